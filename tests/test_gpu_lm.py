"""Accelerated linear method (Sec. II.B): the Eq. 10 products on the CUDA path.

lm_apply evaluates (H x, S x) over the basis {Psi, Psi^j} from the stored
samples with the Hamiltonian factored as in Eq. 9; the oracle evaluates the
same sums with every Q_{n r s j} built from scratch (fresh amplitudes, fresh
O(n'), explicit Jordan-Wigner signs), itself pinned on the CPU against the
explicit <Psi^i|H|Psi^j>.  The GPU never forms O(n'): it differentiates the
in-place move ratios along x.  Tolerances (relative 2-norm over the n_v + 1
components): FP64 store 1e-10, FP32 store 2e-4.

At the full sizes the oracle cannot follow every sample, so the tests there
use the ansatz's null directions: x along a correlator's own
amplitudes, or along f scaled by 2/N, reproduces Psi itself (Psi^x = Psi),
so its products must equal those of x = e_0 to rounding.
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


CASES = {
    "hubbard4x4_pair": lambda: inputs.workload("hubbard4x4_pair", n_walkers=24, samples_per_walker=6),
    "hubbard4x4_2x2": lambda: inputs.workload("hubbard4x4_2x2", n_walkers=13, samples_per_walker=5),
    "abinitio24": lambda: inputs.workload("abinitio24", n_walkers=8, samples_per_walker=2),
    "hubbard3x2_shared": lambda: inputs.hubbard("s", 3, 2, 2, 2, "pair", seed=31, n_walkers=16,
                                                samples_per_walker=3, shared=True),
    "abinitio10_odd_spin": lambda: inputs.abinitio("t", 10, 5, 3, n_chol=12, seed=33, n_walkers=20,
                                                   samples_per_walker=2),
}


def _setup(wl):
    P = oracle.Problem(wl)
    occ = wl.init_occ.copy()
    step = np.zeros(wl.n_walkers, np.uint64)
    smp, _, _ = P.sample(occ, step, 91, 4, wl.samples_per_walker)
    h = V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=True)
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_measure(h, smp)
    return P, smp, h


@pytest.mark.parametrize("name", list(CASES))
def test_lm_products_match_oracle(name):
    wl = CASES[name]()
    P, smp, h = _setup(wl)
    fac = oracle.lm_factors(wl)
    rng = np.random.default_rng(7)
    nv1 = wl.n_params + 1
    for trial in range(2):
        x = rng.standard_normal(nv1)
        if trial == 1:
            x[0] = 0.0
        H_or, S_or = P.lm_apply(smp, fac, x)
        xd = torch.from_numpy(x).cuda()
        Hx, Sx = V.lm_apply(h, xd, V.VMC_STORE_FP64)
        assert rel(Hx.cpu().numpy(), H_or) <= 1e-10
        assert rel(Sx.cpu().numpy(), S_or) <= 1e-10
        Hx32, Sx32 = V.lm_apply(h, xd, V.VMC_STORE_FP32)
        assert rel(Hx32.cpu().numpy(), H_or) <= 2e-4
        assert rel(Sx32.cpu().numpy(), S_or) <= 2e-4
    h.close()


def test_lm_without_S_and_state_errors():
    wl = CASES["hubbard4x4_pair"]()
    h = V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=False)
    V.vmc_set_params(h, wl.C, wl.f)
    x = torch.zeros(wl.n_params + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(V.VmcError) as e:
        V.lm_apply(h, x, V.VMC_STORE_FP64)          # no samples yet
    assert e.value.code == -9
    P, smp, _ = _setup(wl)
    V.vmc_measure(h, smp)
    with pytest.raises(V.VmcError) as e:
        V.lm_apply(h, x, V.VMC_STORE_FP32)          # FP32 store not kept
    assert e.value.code == -9
    x[0] = 1.0
    Hx, Sx = V.lm_apply(h, x, V.VMC_STORE_FP64, want_S=False)
    assert Sx is None
    H_or, _ = P.lm_apply(smp, oracle.lm_factors(wl), x.cpu().numpy())
    assert rel(Hx.cpu().numpy(), H_or) <= 1e-10
    h.close()


def _null_directions(wl):
    """x with Psi^x = Psi: the amplitudes of the first correlator (Psi is
    linear in them) and f * 2/N (Pf is homogeneous of degree N/2)."""
    nv1 = wl.n_params + 1
    xc = np.zeros(nv1)
    k0 = int(wl.corr_param_off[0])
    k1 = k0 + 4 ** len(wl.corr_sites[0])
    xc[1 + k0:1 + k1] = wl.C[k0:k1]
    xf = np.zeros(nv1)
    xf[1 + wl.n_corr_params:] = wl.f * 2.0 / wl.N
    return xc, xf


# FP64 arithmetic is slow on this GPU, so the FP64 cases run on fewer
# walkers; the FP32 cases run the full workloads (65,536 samples)
@pytest.mark.parametrize("name,prec,tol,nw", [("hubbard8x8_2x3", V.VMC_STORE_FP64, 1e-9, 64),
                                              ("hubbard8x8_2x3", V.VMC_STORE_FP32, 1e-3, None),
                                              ("abinitio24", V.VMC_STORE_FP64, 1e-9, 1024),
                                              ("abinitio24", V.VMC_STORE_FP32, 1e-3, None)])
def test_full_size_null_directions(name, prec, tol, nw):
    wl = inputs.workload(name) if nw is None else inputs.workload(name, n_walkers=nw)
    h = V.vmc_create(wl, walker_precision=V.VMC_FP64 if prec == V.VMC_STORE_FP64 else V.VMC_FP32,
                     keep_fp64_store=prec == V.VMC_STORE_FP64, keep_lowp_store=prec == V.VMC_STORE_FP32,
                     refresh_every=1)
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, 10, inputs.seed_sampling_for(name))
    nv1 = wl.n_params + 1
    e0 = torch.zeros(nv1, dtype=torch.float64, device="cuda")
    e0[0] = 1.0
    H0, S0 = V.lm_apply(h, e0, prec)
    H0, S0 = H0.cpu().numpy(), S0.cpu().numpy()
    assert S0[0] == pytest.approx(1.0, rel=1e-12)
    for x in _null_directions(wl):
        Hx, Sx = V.lm_apply(h, torch.from_numpy(x).cuda(), prec)
        assert rel(Sx.cpu().numpy(), S0) <= tol
        assert rel(Hx.cpu().numpy(), H0) <= tol
    h.close()


def _dense(P, smp, fac, nv1):
    H = np.zeros((nv1, nv1))
    S = np.zeros((nv1, nv1))
    for j in range(nv1):
        e = np.zeros(nv1)
        e[j] = 1.0
        H[:, j], S[:, j] = P.lm_apply(smp, fac, e)
    return H, S


@pytest.mark.parametrize("name,nw,spw", [("hubbard3x2_pair", 256, 2), ("abinitio6", 256, 2)])
def test_lm_solve_matches_dense_eigensolver(name, nw, spw):
    """lm_solve (Davidson on the GPU products) against the lowest eigenpair of
    the oracle's dense matrices (one oracle product per column)."""
    import scipy.linalg
    if name == "hubbard3x2_pair":
        wl = inputs.hubbard("t", 3, 2, 2, 2, "pair", seed=9, n_walkers=nw, samples_per_walker=spw)
    else:
        wl = inputs.abinitio("t", 6, 3, 3, n_chol=6, seed=35, n_walkers=nw, samples_per_walker=spw)
    P, smp, h = _setup(wl)
    fac = oracle.lm_factors(wl)
    nv1 = wl.n_params + 1
    H, S = _dense(P, smp, fac, nv1)
    a_shift, eps = 1.0, 1e-2
    D = np.eye(nv1)
    D[0, 0] = 0.0
    lam, vec = scipy.linalg.eigh(0.5 * (H + H.T) + a_shift * D, 0.5 * (S + S.T) + eps * D)
    ref = vec[:, 0] / vec[0, 0]
    x, info = V.lm_solve(h, a_shift, eps, 1e-10, max_iter=2000, max_sub=40, store=V.VMC_STORE_FP64)
    assert info["converged"] == 1
    assert info["eigenvalue"] == pytest.approx(lam[0], rel=1e-8)
    xs = x.cpu().numpy()
    assert rel(xs, ref) <= 1e-5
    assert info["Sx0"] == pytest.approx((S @ xs)[0], rel=1e-9)
    # the update: alpha += x_{1:} / Sx0 on the device
    alpha0 = np.concatenate([wl.C, wl.f])
    V.lm_update(h, x, info["Sx0"])
    C, f = V.vmc_get_params(h)
    assert rel(np.concatenate([C, f]), oracle.lm_update(alpha0, xs, info["Sx0"])) <= 1e-14
    # FP32 store: same eigenvalue to FP32 accuracy
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_measure(h, smp)
    x32, info32 = V.lm_solve(h, a_shift, eps, 1e-6, max_iter=2000, max_sub=40, store=V.VMC_STORE_FP32,
                             allow_not_converged=True)
    assert info32["eigenvalue"] == pytest.approx(lam[0], rel=1e-4)
    h.close()


def test_lm_optimize_lowers_the_energy():
    """Linear-method steps from random parameters on the 4x4 lattice, with
    the energy check of Sec. II.B (a step that raises the energy is undone
    and retried with a larger shift): the accepted steps lower the sampled
    energy well beyond its statistical error, and none raises it."""
    wl = inputs.workload("hubbard4x4_pair", n_walkers=1024, samples_per_walker=4)
    h = V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=False)
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, 20, 5)
    hist = V.lm_optimize(h, 5, 1.0, 1e-2, 1e-6, store=V.VMC_STORE_FP64, seed=11, max_iter=600, max_sub=32)
    acc = [r for r in hist if r["accepted"]]
    assert acc
    e0, err0 = hist[0]["energy"][0], hist[0]["energy"][2]     # mean, variance, standard error
    e1, err1 = acc[-1]["energy_after"][0], acc[-1]["energy_after"][2]
    assert e1 < e0 - 5 * max(err0, err1)
    h.close()


def test_lm_rank_local_products_add_up():
    """Two handles holding 1/3 and 2/3 of the samples: their sample-count
    weighted products (what the sharded solve all-reduces) equal the product
    of one handle holding all samples."""
    from paper_1108_0900_gb300 import shard
    wl = CASES["abinitio10_odd_spin"]()
    P, smp, h = _setup(wl)
    cut = len(smp) // 3
    parts = []
    for sl in (slice(0, cut), slice(cut, None)):
        hp = V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=False)
        V.vmc_set_params(hp, wl.C, wl.f)
        V.vmc_measure(hp, np.ascontiguousarray(smp[sl]))
        parts.append(hp)
    x = torch.from_numpy(np.random.default_rng(4).standard_normal(wl.n_params + 1)).cuda()
    locs = [shard.LibraryLocal(hp, V.VMC_STORE_FP64) for hp in parts]
    res = [loc.lm_product(x) for loc in locs]
    N = sum(n for _, _, n in res)
    Hx = sum(H * n for H, _, n in res) / N
    Sx = sum(S * n for _, S, n in res) / N
    H_all, S_all = V.lm_apply(h, x, V.VMC_STORE_FP64)
    assert rel(Hx.cpu().numpy(), H_all.cpu().numpy()) <= 1e-12
    assert rel(Sx.cpu().numpy(), S_all.cpu().numpy()) <= 1e-12
    for hp in parts:
        hp.close()
    h.close()
