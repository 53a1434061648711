"""Lattices of uneven size in one launch: an 8x8 lattice with 28 + 28
electrons and 2x2 plaquettes together with a 4x4 lattice with 8 + 8
electrons and bond pairs.  Batched sampling must give every handle exactly
the samples of its own vmc_sample with the same seed (integers bit-exact,
floating point bit-exact: the same arithmetic per walker), and the batched
S product must equal each handle's own product (1e-12, FP64; the CTAs are
split differently, so only the summation order differs) and the oracle's
Eq. 7 of the stored rows (1e-10)."""
import numpy as np
import pytest

import oracle
from pair_blocks import block_pairs
from paper_1108_0900_gb300 import inputs
from paper_1108_0900_gb300 import vmcsr as V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


def _pair(prec, keep64=True):
    wa = inputs.workload("hubbard8x8_2x2", n_walkers=64, samples_per_walker=3)
    wb = inputs.workload("hubbard4x4_pair", n_walkers=96, samples_per_walker=4)
    hs = []
    for w in (wa, wb):
        h = V.vmc_create(w, walker_precision=prec, keep_fp64_store=keep64, keep_lowp_store=True)
        V.vmc_set_params(h, w.C, w.f)
        V.vmc_set_walkers(h, w.init_occ)
        hs.append(h)
    return (wa, wb), hs


@pytest.mark.parametrize("prec", [V.VMC_FP64, V.VMC_FP32])
def test_batched_sampling_equals_separate_runs(prec):
    wls, batch = _pair(prec)
    _, solo = _pair(prec)
    seeds = [101, 202]
    V.vmc_sample_batch(batch, 3, seeds)
    for h, sd in zip(solo, seeds):
        V.vmc_sample(h, 3, sd)
    store = V.VMC_STORE_FP64
    for hb, hs in zip(batch, solo):
        a = V.vmc_get_samples(hb, store)
        b = V.vmc_get_samples(hs, store)
        for u, v in zip(a, b):
            assert np.array_equal(u, v)
        oa, sa = V.vmc_get_walkers(hb)
        ob, sb = V.vmc_get_walkers(hs)
        assert np.array_equal(oa, ob) and np.array_equal(sa, sb)
    for h in batch + solo:
        h.close()


def test_batched_product_equals_own_products_and_oracle():
    wls, hs = _pair(V.VMC_FP64)
    V.vmc_sample_batch(hs, 3, [7, 8])
    rng = np.random.default_rng(4)
    Vs = [torch.from_numpy(rng.standard_normal(w.n_params)).cuda() for w in wls]
    for store in (V.VMC_STORE_FP64, V.VMC_STORE_FP32):
        for h in hs:
            V.sr_gradient(h, store)
        outs = V.sr_apply_S_batch(hs, Vs, wls[0].shift, store)
        for h, w, v, o in zip(hs, wls, Vs, outs):
            own = V.sr_apply_S(h, v, w.shift, store).cpu().numpy()
            assert rel(o.cpu().numpy(), own) <= 1e-12
            if store == V.VMC_STORE_FP64:
                occ, _, cs, pf = V.vmc_get_samples(h, V.VMC_STORE_FP64)
                ref, _ = oracle.apply_S_compact(oracle.Problem(w), occ, cs, block_pairs(w.n_up, w.n_dn), pf,
                                                v.cpu().numpy(), w.shift)
                assert rel(o.cpu().numpy(), ref) <= 1e-10
    for h in hs:
        h.close()


def test_batched_calls_reject_bad_arguments():
    wls, hs = _pair(V.VMC_FP64)
    with pytest.raises(V.VmcError):
        V.vmc_sample_batch([hs[0], hs[0]], 0, [1, 2])         # a handle twice
    h32 = V.vmc_create(wls[1], walker_precision=V.VMC_FP32, keep_fp64_store=True, keep_lowp_store=False)
    V.vmc_set_params(h32, wls[1].C, wls[1].f)
    V.vmc_set_walkers(h32, wls[1].init_occ)
    with pytest.raises(V.VmcError):
        V.vmc_sample_batch([hs[0], h32], 0, [1, 2])           # mixed walker precisions
    with pytest.raises(V.VmcError):
        V.sr_apply_S_batch(hs, [torch.zeros(w.n_params, dtype=torch.float64, device="cuda") for w in wls],
                           1e-3, V.VMC_STORE_BF16)            # BF16 is not a batched store
    for h in hs + [h32]:
        h.close()
