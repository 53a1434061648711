"""FP32 walkers with the FP64 refresh of their stored samples, the chains'
log-amplitude drift, and the mixed solve against the FP64 operator.

The FP32 chains (ratios, rank-2 inverse updates) decide the Markov walk;
with fp64_refresh every stored sample is then evaluated from scratch in FP64
(pairing inverse, E_L, O), so the stores hold the FP64 values (rounded to
FP32 / BF16 where stored so) and agree with the oracle to FP64 precision on
the same configurations.  Tolerances: E_L and the FP64 store 1e-10 (as every
FP64 stage), the FP32 store 1e-7 (one rounding, 2^-24); without the refresh
the FP32 walkers' own values carry the FP32 inversion error (about
u_32 kappa(A)), up to 5e-3 on these configurations.  VMC_CG_MIXED64 streams
BF16 in the inner solve and reports the true residual against the FP64
operator, which must meet the tolerance (1e-6).
"""
import numpy as np
import pytest

import oracle
from paper_1108_0900_gb300 import inputs
from paper_1108_0900_gb300 import vmcsr as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


def pf_index(M, p, q):
    return p * M - p * (p + 1) // 2 + (q - p - 1)


def _oracle_rows(wl, P, occ):
    from pair_blocks import block_pairs
    E, O = P.measure(occ)
    pl = block_pairs(wl.n_up, wl.n_dn)
    p = occ[:, pl[:, 0]].astype(np.int64)
    q = occ[:, pl[:, 1]].astype(np.int64)
    pf = np.take_along_axis(O, wl.n_corr_params + pf_index(wl.M, p, q), axis=1)
    return E, pf


@pytest.mark.parametrize("name,nw,spw", [("hubbard8x8_2x3", 128, 4), ("abinitio24", 64, 4), ("hubbard4x4_2x2", 256, 4)])
def test_fp64_refresh_matches_the_oracle(name, nw, spw):
    wl = inputs.workload(name, n_walkers=nw, samples_per_walker=spw)
    h = V.vmc_create(wl, walker_precision=V.VMC_FP32, keep_fp64_store=True, keep_lowp_store=True, fp64_refresh=True)
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, 3, inputs.seed_sampling_for(name))
    occ, E, cs, pf64 = V.vmc_get_samples(h, V.VMC_STORE_FP64)
    _, _, _, pf32 = V.vmc_get_samples(h, V.VMC_STORE_FP32)
    P = oracle.Problem(wl)
    pick = np.random.default_rng(3).choice(len(occ), 24, replace=False)
    E_or, pf_or = _oracle_rows(wl, P, occ[pick])
    for j, s in enumerate(pick):
        assert abs(E[s] - E_or[j]) <= 1e-10 * max(1.0, abs(E_or[j]))
        assert rel(pf64[s], pf_or[j]) <= 1e-10
        assert rel(pf32[s], pf_or[j]) <= 1e-7
    st = V.vmc_sample_stats(h)
    assert st["refreshed"] == 1
    # the FP32 chains' own drift and E_L error are measured, not bounded
    # here: they grow with kappa(A) of the walkers' pairing blocks
    assert np.isfinite(st["lnpsi_drift_max"]) and 0.0 <= st["lnpsi_drift_mean"] <= st["lnpsi_drift_max"]
    assert np.isfinite(st["el_refresh_change_max"]) and st["el_refresh_change_max"] > 0.0
    print(name, st)
    h.close()


def test_running_log_amplitude_of_fp64_chains_is_exact():
    """FP64 chains: the running sum of ln|ratio| over accepted moves equals
    the change of ln|Psi| from scratch (Parlett-Reid pfaffian) to 1e-9."""
    wl = inputs.workload("hubbard4x4_2x2", n_walkers=64, samples_per_walker=6)
    h = V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=False)
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, 2, 77)
    st = V.vmc_sample_stats(h)
    assert st["refreshed"] == 0
    assert st["lnpsi_drift_max"] <= 1e-9
    h.close()


def test_mixed64_residual_against_the_fp64_operator():
    """FP32 walkers with the FP64 refresh on the 8x8 / 2x3 lattice: the mixed
    solve with the FP64-store outer iteration meets 1e-6 against the FP64
    operator, checked again here with an independent FP64 product."""
    wl = inputs.workload("hubbard8x8_2x3", n_walkers=2048, samples_per_walker=4)
    h = V.vmc_create(wl, walker_precision=V.VMC_FP32, keep_fp64_store=True, keep_lowp_store=True, fp64_refresh=True)
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, 4, inputs.seed_sampling_for("hubbard8x8_2x3"))
    g, _ = V.sr_gradient(h, V.VMC_STORE_FP64)
    x, info = V.sr_cg_solve(h, g, wl.shift, 1e-6, 40000, V.VMC_CG_MIXED64)
    assert info["converged"] and info["true_rel_residual"] <= 1e-6
    Sx = V.sr_apply_S(h, x, wl.shift, V.VMC_STORE_FP64)
    res = (torch.linalg.norm(g - Sx) / torch.linalg.norm(g)).item()
    assert res <= 1e-6, res
    h.close()
