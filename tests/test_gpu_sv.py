"""The BF16 S product (Eq. 7) against the oracle's exact Eq. 7 of the same
stored values, and the bounded waits of the staged products.

The BF16 store rounds O once (2^-9); every later step of the product runs in
FP32 with FP64 scalars.  So the CUDA product is compared with the FP64 Eq. 7
of the very values the store holds (read back through vmc_get_samples), and
the only error left is FP32 accumulation: 2e-5 relative (2-norm) to the
larger of the result and the covariance's mean term, the bound written below.  One-vector products run the fused single pass over the
sorted rows; two- and four-vector products the sorted two-pass product.
Geometries cover 16, 24 and 64 sites, shared correlator blocks, 9-site
correlators (32-bit states), ragged sample counts, and the full
65,536-sample 8x8 / 2x3-plaquette store of the benchmark.
"""
import numpy as np
import pytest

import oracle
from pair_blocks import block_pairs
from paper_1108_0900_gb300 import inputs
from paper_1108_0900_gb300 import vmcsr as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_BF16_EXACT = 2e-5


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


def _handle(wl, prec=V.VMC_FP64):
    h = V.vmc_create(wl, walker_precision=prec, keep_fp64_store=False, keep_lowp_store=True)
    V.vmc_set_params(h, wl.C, wl.f)
    return h


# product paths checked per number of vectors (a path that does not apply
# to a problem falls back to the next one, which is then checked again)
PATHS = {1: (V.VMC_PATH_SORTED, V.VMC_PATH_FUSED, V.VMC_PATH_STAGED, V.VMC_PATH_GENERIC, V.VMC_PATH_COMPACT),
         2: (V.VMC_PATH_SORTED, V.VMC_PATH_STAGED),
         4: (V.VMC_PATH_SORTED, V.VMC_PATH_GENERIC)}


def _check_products(wl, h, ks=(1, 2, 4), seed=8, paths=PATHS):
    V.sr_gradient(h, V.VMC_STORE_BF16)
    occ, _, cs, pf = V.vmc_get_samples(h, V.VMC_STORE_BF16)
    P = oracle.Problem(wl)
    pairs = block_pairs(wl.n_up, wl.n_dn)
    rng = np.random.default_rng(seed)
    for k in ks:
        v = rng.standard_normal((k, wl.n_params))
        ref, Obar = oracle.apply_S_compact(P, occ, cs, pairs, pf, v, wl.shift)
        for path in paths[k]:
            V.vmc_set_product_path(h, path)
            out = V.sr_apply_S(h, torch.from_numpy(v).cuda(), wl.shift, V.VMC_STORE_BF16).cpu().numpy()
            for j in range(k):
                # FP32 rounding is relative to the operands of the covariance, whose
                # mean term |Obar| |Obar . v| can exceed the result (with one sample
                # S = 0 and the exact result is shift v)
                scale = max(np.linalg.norm(ref[j]), np.linalg.norm(Obar) * abs(Obar @ v[j]))
                err = np.linalg.norm(out[j] - ref[j]) / scale
                assert err <= TOL_BF16_EXACT, (k, V.PATH_NAMES[path], j, err)
    V.vmc_set_product_path(h, V.VMC_PATH_AUTO)


GEOMETRIES = {
    # 16 sites
    "hubbard4x4_pair": lambda: inputs.workload("hubbard4x4_pair", n_walkers=64, samples_per_walker=8),
    "hubbard4x4_2x2": lambda: inputs.workload("hubbard4x4_2x2", n_walkers=301, samples_per_walker=3),
    # 24 sites
    "abinitio24": lambda: inputs.workload("abinitio24", n_walkers=97, samples_per_walker=3),
    # 64 sites, 4,096-state correlators
    "hubbard8x8_2x2": lambda: inputs.workload("hubbard8x8_2x2", n_walkers=211, samples_per_walker=2),
    "hubbard8x8_2x3": lambda: inputs.workload("hubbard8x8_2x3", n_walkers=257, samples_per_walker=2),
    # every plaquette on one block of 4,096 amplitudes
    "hubbard8x8_2x3_shared": lambda: inputs.hubbard("s5", 8, 8, 28, 28, "2x3", seed=13, n_walkers=129,
                                                    samples_per_walker=3, shared=True),
    # 3x3 correlators, one block of 4^9 per sublattice (18-bit states)
    "paper4x4_3x3": lambda: inputs.hubbard("p33", 4, 4, 8, 8, "3x3", seed=14, n_walkers=133, samples_per_walker=3,
                                           shared=True),
    # fewer electrons than half filling, an odd sample count
    "hubbard8x8_doped_odd": lambda: inputs.hubbard("d", 8, 8, 20, 18, "2x2", seed=17, n_walkers=77,
                                                   samples_per_walker=1),
}


@pytest.mark.parametrize("name", list(GEOMETRIES))
def test_bf16_product_equals_exact_eq7_of_the_store(name):
    wl = GEOMETRIES[name]()
    h = _handle(wl)
    n = wl.n_walkers * wl.samples_per_walker
    cfgs = inputs.draw_configs(np.random.default_rng(11), n, wl.n_sites, wl.n_up, wl.n_dn)
    V.vmc_measure(h, cfgs)
    _check_products(wl, h)
    h.close()


@pytest.mark.parametrize("n", [1, 2, 3, 7, 913, 8193, 20001])
def test_bf16_product_ragged_sample_counts(n):
    """One sample (S = 0: the result is shift v), two, three, seven (one warp
    of the single pass with a sample more than the others), a count that
    leaves the CTAs of the pass with unequal shares, and counts past one
    8,192-sample chunk of the parameter-major copy (one sample in the second
    chunk; two full chunks and a ragged third), whose per-chunk sums the
    scatter adds up; those also for two and four vectors."""
    wl = inputs.workload("hubbard8x8_2x3", n_walkers=n, samples_per_walker=1)
    h = _handle(wl)
    cfgs = inputs.draw_configs(np.random.default_rng(n), n, wl.n_sites, wl.n_up, wl.n_dn)
    V.vmc_measure(h, cfgs)
    _check_products(wl, h, ks=(1,) if n < 8192 else (1, 2, 4))
    h.close()


def test_bf16_product_full_size_benchmark_store():
    """The benchmark's store: 16,384 FP32 walkers x 4 samples drawn from
    |Psi|^2 on the 8x8 lattice with 64 2x3 plaquettes (n_v = 270,272); the
    single pass (one vector) and the sorted pass (four vectors) against the
    exact Eq. 7 of all 65,536 stored rows."""
    wl = inputs.workload("hubbard8x8_2x3")
    h = _handle(wl, prec=V.VMC_FP32)
    V.vmc_set_walkers(h, wl.init_occ)
    V.vmc_sample(h, 4, inputs.seed_sampling_for("hubbard8x8_2x3"))
    assert V.vmc_num_samples(h) == 65536
    _check_products(wl, h, ks=(1, 4), paths={1: (V.VMC_PATH_SORTED, V.VMC_PATH_FUSED, V.VMC_PATH_COMPACT),
                                              4: (V.VMC_PATH_SORTED,)})
    h.close()


def test_autotune_picks_a_measured_path_and_keeps_parity(tmp_path):
    """sr_autotune times every applicable path and makes the fastest the
    AUTO choice; the tuned products still equal the exact Eq. 7; the JSON
    cache gives the same choice back without timing."""
    wl = inputs.workload("hubbard8x8_2x3", n_walkers=2048, samples_per_walker=2)
    h = _handle(wl)
    cfgs = inputs.draw_configs(np.random.default_rng(21), 4096, wl.n_sites, wl.n_up, wl.n_dn)
    V.vmc_measure(h, cfgs)
    V.sr_gradient(h, V.VMC_STORE_BF16)
    res = V.sr_autotune(h, reps=3)
    # (four pairing images of 8,128 amplitudes exceed shared memory, so the
    # generic pass does not apply to four vectors here)
    assert set(res["ms"]) >= {"sorted", "fused", "generic", "compact"} and "sorted" in res["ms4"]
    assert res["ms"][res["path"]] == min(res["ms"].values())
    assert res["ms4"][res["path4"]] == min(res["ms4"].values())
    _check_products(wl, h, ks=(1, 4), paths={1: (V.VMC_PATH_AUTO,), 4: (V.VMC_PATH_AUTO,)})
    cache = str(tmp_path / "tune.json")
    first = V.tuned(h, cache, "hubbard8x8_2x3:4096", reps=2)
    h2 = _handle(wl)
    V.vmc_measure(h2, cfgs)
    again = V.tuned(h2, cache, "hubbard8x8_2x3:4096")
    assert again["cached"] and not first["cached"]
    assert (again["path"], again["path4"]) == (first["path"], first["path4"])
    _check_products(wl, h2, ks=(1,), paths={1: (V.VMC_PATH_AUTO,)})
    h.close()
    h2.close()


def test_staged_wait_limit_reports_timeout_and_recovers():
    """The FP32-store product stages every sample in shared memory with bulk
    copies and waits on an mbarrier a bounded number of times.
    vmc_set_wait_limit(h, 0) makes its first wait give up before the copy
    lands: the kernel drains its copies and the call returns VMC_ERR_TIMEOUT
    (no fault, no hang).  With the default limit the same handle then gives
    the same products again, and the BF16 product (which stages nothing)
    is unaffected by the limit: the context is intact."""
    wl = inputs.workload("hubbard8x8_2x3", n_walkers=300, samples_per_walker=2)
    h = _handle(wl)
    cfgs = inputs.draw_configs(np.random.default_rng(5), 600, wl.n_sites, wl.n_up, wl.n_dn)
    V.vmc_measure(h, cfgs)
    V.sr_gradient(h, V.VMC_STORE_BF16)
    v = torch.from_numpy(np.random.default_rng(6).standard_normal(wl.n_params)).cuda()
    ref = V.sr_apply_S(h, v, wl.shift, V.VMC_STORE_BF16).cpu().numpy()
    ref32 = V.sr_apply_S(h, v, wl.shift, V.VMC_STORE_FP32_F32ACC).cpu().numpy()
    V.vmc_set_wait_limit(h, 0)
    with pytest.raises(V.VmcError) as e:
        V.sr_apply_S(h, v, wl.shift, V.VMC_STORE_FP32_F32ACC)
    assert e.value.code == -6
    assert rel(V.sr_apply_S(h, v, wl.shift, V.VMC_STORE_BF16).cpu().numpy(), ref) <= 1e-6
    V.vmc_set_wait_limit(h, 1 << 22)
    again = V.sr_apply_S(h, v, wl.shift, V.VMC_STORE_BF16).cpu().numpy()
    again32 = V.sr_apply_S(h, v, wl.shift, V.VMC_STORE_FP32_F32ACC).cpu().numpy()
    # (the correlator sums add float atomics in no fixed order: 1e-6, not bits)
    assert rel(again, ref) <= 1e-6
    assert rel(again32, ref32) <= 1e-6
    # a CG solve on the same handle converges as usual
    g, _ = V.sr_gradient(h, V.VMC_STORE_FP32)
    _, info = V.sr_cg_solve(h, g, wl.shift, 1e-6, 20000, V.VMC_CG_MIXED)
    assert info["converged"]
    h.close()
