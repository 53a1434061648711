"""The allocation-free pairing-block product, sr_pairing_product_noalloc.

It serves callers that cannot call cudaMalloc (a pool allocator already owns
the device memory, or the caller is in a latency-critical loop where
cudaMalloc would synchronise the device).  Its scratch is a fixed device
array inside the library.  This file runs last so that, if it fails, a run
that stops at the first failure has already run every other test.

The result is checked against the existing entry points on the same samples:
sr_apply_S (FP32 store, FP32 accumulation) gives
(1/n_s) sum_s t_s O_s - Obar (Obar . v) on the pairing block, and
vmc_logpsi_backward with unit weights gives n_s Obar, so
n_s (S v + Obar (Obar . v)) restricted to the pairing block must equal the
allocation-free sum_s t_s O_s.  Tolerance: the 1e-5 of FP32 S products.
"""
import numpy as np
import pytest

from paper_1108_0900_gb300 import inputs
from paper_1108_0900_gb300 import vmcsr as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _pair_index(wl, occ):
    M, nu, N = wl.M, wl.n_up, wl.N
    pl = [(a, b) for a in range(nu) for b in range(a + 1, nu)]
    pl += [(a, b) for a in range(nu, N) for b in range(a + 1, N)]
    pl += [(a, b) for a in range(nu) for b in range(nu, N)]
    a = np.array([x for x, _ in pl])
    b = np.array([y for _, y in pl])
    p = occ[:, a].astype(np.int64)
    q = occ[:, b].astype(np.int64)
    return p * M - p * (p + 1) // 2 + (q - p - 1)


@pytest.mark.parametrize("name,nw,spw", [("hubbard8x8_2x3", 1024, 4), ("hubbard4x4_pair", 64, 8)])
def test_noalloc_matches_existing_entry_points(name, nw, spw):
    wl = inputs.workload(name, n_walkers=nw, samples_per_walker=spw)
    h = V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=True)
    V.vmc_set_params(h, wl.C, wl.f)
    cfgs = inputs.draw_configs(np.random.default_rng(77), nw * spw, wl.n_sites, wl.n_up, wl.n_dn)
    V.vmc_measure(h, cfgs)
    occ, _, _, pf = V.vmc_get_samples(h, V.VMC_STORE_FP32)
    n = len(occ)
    npf = wl.n_pf_params
    occ_d = torch.from_numpy(occ).cuda()
    pf_d = torch.from_numpy(pf.astype(np.float32)).cuda()
    v = np.random.default_rng(5).standard_normal(npf).astype(np.float32)
    v_d = torch.from_numpy(v).cuda()

    # existing entry points
    Vfull = np.zeros(wl.n_params)
    Vfull[wl.n_corr_params:] = v
    Sv = V.sr_apply_S(h, torch.from_numpy(Vfull).cuda(), 0.0, V.VMC_STORE_FP32_F32ACC).cpu().numpy()
    Osum = V.vmc_logpsi_backward(h, torch.ones(n, dtype=torch.float64)).cpu().numpy()
    Obar = Osum / n
    expect = n * (Sv + Obar * (Obar @ Vfull))[wl.n_corr_params:]
    # per-sample dots from the stored values
    pq = _pair_index(wl, occ)
    t_expect = (pf.astype(np.float32).astype(np.float64) * v.astype(np.float64)[pq]).sum(1)

    for call in range(2):
        t, out = V.sr_pairing_product_noalloc(wl.n_sites, wl.n_up, wl.n_dn, occ_d, pf_d, v_d)
        torch.cuda.synchronize()
        out = out.cpu().numpy()
        t = t.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(out - expect) <= 1e-5 * np.linalg.norm(expect), call
        assert np.linalg.norm(t - t_expect) <= 1e-5 * np.linalg.norm(t_expect), call
    h.close()


def test_noalloc_rejects_oversized_and_bad_strides():
    occ = torch.zeros((4, 2), dtype=torch.uint8, device="cuda")
    pf = torch.zeros((4, 1), dtype=torch.float32, device="cuda")
    v = torch.zeros(65 * 2 * (65 * 2 - 1) // 2, dtype=torch.float32, device="cuda")
    with pytest.raises(V.VmcError) as e:
        V.sr_pairing_product_noalloc(65, 1, 1, occ, pf, v)     # 65 sites: beyond the fixed scratch
    assert e.value.code == -1 and "scratch" in str(e.value)
    with pytest.raises(V.VmcError) as e:
        V.sr_pairing_product_noalloc(4, 2, 2, occ, pf, v)      # rows shorter than N / P
    assert e.value.code == -1


def test_noalloc_skips_occupations_outside_the_sector():
    """A caller-given occupation that is not a configuration of the sector
    (an orbital beyond M, a repeated orbital, an up electron in the down
    block) would index outside the pairing images; the kernel checks every
    sample, gives it t_s = NaN and leaves it out of the sum, so the result
    equals the product over the valid samples alone."""
    wl = inputs.workload("hubbard4x4_pair", n_walkers=8, samples_per_walker=4)
    n = 32
    cfgs = inputs.draw_configs(np.random.default_rng(3), n, wl.n_sites, wl.n_up, wl.n_dn)
    P = wl.n_up * (wl.n_up - 1) // 2 + wl.n_dn * (wl.n_dn - 1) // 2 + wl.n_up * wl.n_dn
    pf = np.random.default_rng(4).standard_normal((n, P)).astype(np.float32)
    v = np.random.default_rng(5).standard_normal(wl.n_pf_params).astype(np.float32)
    bad = cfgs.copy()
    bad[3, -1] = 2 * wl.n_sites + 5          # orbital beyond M - 1
    bad[7, 1] = bad[7, 0]                    # repeated orbital (not ascending)
    bad[11, 0] = wl.n_sites                  # an up electron in the down block
    bad[11] = np.sort(bad[11])
    good = np.setdiff1d(np.arange(n), [3, 7, 11])
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    t_all, out_all = V.sr_pairing_product_noalloc(wl.n_sites, wl.n_up, wl.n_dn, to(bad), to(pf), to(v))
    t_good, out_good = V.sr_pairing_product_noalloc(wl.n_sites, wl.n_up, wl.n_dn, to(bad[good]), to(pf[good]),
                                                     to(v))
    torch.cuda.synchronize()
    t_all = t_all.cpu().numpy()
    assert np.isnan(t_all[[3, 7, 11]]).all()
    assert np.isfinite(t_all[good]).all()
    assert np.array_equal(t_all[good], t_good.cpu().numpy())
    o1, o2 = out_all.cpu().numpy(), out_good.cpu().numpy()
    assert np.linalg.norm(o1 - o2) <= 1e-5 * np.linalg.norm(o2)
