#!/usr/bin/env python
"""SR-iteration benchmark of the matrix-free SR hot path on one GB300.

One step = one stochastic-reconfiguration iteration of the 8x8 periodic
Hubbard workload (28 + 28 electrons, 64 2x3-plaquette correlators + pfaffian,
270,272 parameters, 16,384 walkers x 4 samples = 65,536 samples):
  vmc_sample (4 sweeps per walker, chains continue from the previous step)
  -> sr_gradient -> sr_cg_solve to relative residual 1e-6.
The mixed path (FP32 walkers, BF16 O stream with FP32 accumulation, FP64
scalars and FP64-accumulated residuals) is the headline; the plain FP64 path
runs the same step for comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With torchrun (N > 1) every rank runs an independent replica (different
sampling seed); the reported time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SR-iteration s and S·v GB/s, mixed vs FP64 on 1 GB300 at rel. residual 1e-6"
WORKLOAD = ("8x8 periodic Hubbard U/t=4, 28+28 electrons, 64 2x3-plaquette correlators + pfaffian over 128 "
            "spin orbitals (n_v=270,272), 16,384 walkers x 4 samples = 65,536 samples, shift 1e-3, CG to 1e-6")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 5 + i and r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

# DRAM bytes per BF16 product on this workload, counted by ncu
# (dram__bytes_read + dram__bytes_write, one capture per path): the sorted
# two-pass product reads G (429 MB with its writes) and T in 8,192-sample
# chunks with the correlator states (446 MB); the fused single pass reads G
# once (430 MB) plus the per-CTA images and the correlator states in its
# finish (23 MB).
PASS_DRAM_BYTES = {"sorted": 875.0e6, "fused": 453.0e6}
PASS_KERNELS = {"sorted": "k_gather_G<1,U> + k_scatter_T<1> (sorted two-pass Eq. 7 product, BF16 store)",
                "compact": "k_gather_C<U> + k_scatter_T<1> (two-pass Eq. 7 product, compact gather, BF16 store)",
                "fused": "k_sv_fused<U> + k_sv_finish (fused single-pass Eq. 7 product, BF16 store)",
                "staged": "k_sr_stream<bf16,1> + k_corr_scatter + k_reduce_pf (staged per-sample pass)",
                "generic": "k_sr_main<bf16,float,1> + k_corr_scatter + k_reduce_pf (generic per-sample pass)"}
# nominal FP64 (non-tensor) rate of one GB300 (the peaks file measures no FP64)
FP64_PEAK_TFLOPS = 1.25
AUTOTUNE_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1108_0900_gb300", "_build",
                              "autotune.json")


def run_gpu(args, rank, world, dist):
    import torch
    from paper_1108_0900_gb300 import inputs
    from paper_1108_0900_gb300 import vmcsr as V

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    wl = inputs.workload("hubbard8x8_2x3")
    seed = inputs.seed_sampling_for("hubbard8x8_2x3") + 7919 * rank
    shift, tol = wl.shift, 1e-6
    max_iter = 20000

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def make(path, w=None):
        w = w or wl
        prec = V.VMC_FP64 if path == "fp64" else V.VMC_FP32
        h = V.vmc_create(w, walker_precision=prec, keep_fp64_store=path in ("fp64", "refresh64"),
                         keep_lowp_store=path != "fp64", fp64_refresh=path == "refresh64")
        V.vmc_set_params(h, w.C, w.f)
        V.vmc_set_walkers(h, w.init_occ)
        V.vmc_sample(h, w.burn_in_sweeps, seed)       # thermalisation, outside every timed region
        return h

    def step(h, path, k, info_out):
        V.vmc_sample(h, 0, seed + 1 + k)
        store = V.VMC_STORE_FP64 if path in ("fp64", "refresh64") else V.VMC_STORE_FP32
        g, _ = V.sr_gradient(h, store, stats=False)
        mode = {"mixed": V.VMC_CG_MIXED, "block4": V.VMC_CG_BLOCK4,
                "refresh64": V.VMC_CG_MIXED64}.get(path, V.VMC_CG_FP64)
        x, info = V.sr_cg_solve(h, g, shift, tol, max_iter, mode, allow_not_converged=True)
        info_out.append(info)
        return x

    def timed(h, path, steps, warmup, profile=False, store=None):
        infos = []
        for k in range(warmup):
            step(h, path, k, infos)
        barrier()
        infos.clear()
        if profile:
            V.vmc_profile(h, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with Clocks(local) as clk:
            e0.record()
            for k in range(steps):
                step(h, path, warmup + k, infos)
            e1.record()
            barrier()
        ms = e0.elapsed_time(e1) / steps
        if store is None:
            store = V.VMC_STORE_FP64 if path == "fp64" else V.VMC_STORE_BF16
        prof = V.vmc_profile_read(h, store) if profile else None
        if profile:
            V.vmc_profile(h, False)
        return ms, infos, prof, clk.summary()

    def tune(h, key):
        V.vmc_sample(h, 0, seed + 991)
        V.sr_gradient(h, V.VMC_STORE_BF16, stats=False)
        return V.tuned(h, AUTOTUNE_CACHE, key)

    # ---- mixed path (headline) ----------------------------------------------
    hm = make("mixed")
    tuning = tune(hm, f"hubbard8x8_2x3:{wl.n_samples}")
    ms, infos, prof, clocks = timed(hm, "mixed", args.steps, args.warmup, profile=True)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # ---- the same step with the enlarged block CG (four parameter-group
    # columns, four-vector BF16 products) as the inner solve ----------------
    block = None
    if args.block_steps > 0:
        ms_b, infos_b, prof_b, _ = timed(hm, "block4", args.block_steps, 1, profile=True)
        block = {"ms_per_step": round(ms_b, 3),
                 "inner_block_iterations": float(np.mean([i["iterations"] for i in infos_b])),
                 "outer_steps": float(np.mean([i["refinements"] for i in infos_b])),
                 "four_vector_product_ms": round(prof_b["pass_ms"] / max(1, prof_b["pass_launches"]), 4)
                 if prof_b and prof_b["pass_launches"] else None,
                 "true_rel_residual": max(i["true_rel_residual"] for i in infos_b),
                 "converged": all(i["converged"] for i in infos_b)}

    # ---- the same step with the FP64 refresh of the stored samples and the
    # mixed solve reporting its residual against the FP64 operator -----------
    refresh = None
    if args.refresh_steps > 0:
        hr = make("refresh64")
        ms_r, infos_r, _, _ = timed(hr, "refresh64", args.refresh_steps, 1)
        st = V.vmc_sample_stats(hr)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record()
        V.vmc_sample(hr, 0, seed + 4242)
        e1.record()
        barrier()
        ms_walk_r = e0.elapsed_time(e1)
        refresh = {"ms_per_step": round(ms_r, 3),
                   "sample_with_fp64_refresh_ms": round(ms_walk_r, 3),
                   "cg": "VMC_CG_MIXED64: BF16 inner products, outer iteration and true residual over the FP64 store",
                   "true_rel_residual_vs_fp64_operator": max(i["true_rel_residual"] for i in infos_r),
                   "converged": all(i["converged"] for i in infos_r),
                   "cg_inner_iterations": float(np.mean([i["iterations"] for i in infos_r])),
                   "fp32_chain_lnpsi_drift": {"max": st["lnpsi_drift_max"], "mean": st["lnpsi_drift_mean"]},
                   "fp32_chain_el_error_removed_by_refresh": {"max": st["el_refresh_change_max"],
                                                              "mean": st["el_refresh_change_mean"]}}
        hr.close()

    # ---- end to end through the public API with host buffers ----------------
    import ctypes as ct
    pin_C = torch.from_numpy(wl.C.copy()).pin_memory()
    pin_f = torch.from_numpy(wl.f.copy()).pin_memory()
    x_host = torch.empty(wl.n_params, dtype=torch.float64).pin_memory()
    e2e_ms = []
    barrier()
    for k in range(max(1, args.steps)):
        t0 = time.perf_counter()
        V.vmc_set_params(hm, pin_C.numpy(), pin_f.numpy())        # host -> device parameters
        infos_e2e = []
        x = step(hm, "mixed", 1000 + k, infos_e2e)
        x_host.copy_(x, non_blocking=True)                        # device -> host update
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d = (wl.C.nbytes + wl.f.nbytes)
    d2h = x_host.numel() * 8

    # ---- translation-invariant (shared) correlators, mixed path: every 2x3
    # plaquette of the 8x8 lattice reading one block of 4,096 amplitudes, and
    # the paper's 4x4 layout (a 3x3 correlator at every site, one block of 4^9
    # amplitudes per sublattice, 524,784 parameters) -------------------------
    shared = None
    if args.shared_steps > 0:
        shared = {}
        cases = {
            "8x8_2x3_shared": (inputs.hubbard("8x8-2x3-shared", 8, 8, 28, 28, "2x3", seed=1005, n_walkers=16384,
                                              samples_per_walker=4, shared=True),
                               "8x8 periodic Hubbard U/t=4, 28+28 electrons, 64 2x3 plaquettes sharing one block "
                               "of 4,096 amplitudes + pfaffian"),
            "4x4_3x3_sublattice": (inputs.hubbard("4x4-3x3", 4, 4, 8, 8, "3x3", seed=1006, n_walkers=16384,
                                                  samples_per_walker=4, shared=True),
                                   "4x4 periodic Hubbard U/t=4, 8+8 electrons, a 3x3 correlator at every site "
                                   "sharing one block of 4^9 amplitudes per sublattice + pfaffian"),
        }
        for key, (wls, text) in cases.items():
            hs = V.vmc_create(wls, walker_precision=V.VMC_FP32, keep_fp64_store=False, keep_lowp_store=True)
            V.vmc_set_params(hs, wls.C, wls.f)
            V.vmc_set_walkers(hs, wls.init_occ)
            V.vmc_sample(hs, wls.burn_in_sweeps, seed + 17)
            ms_s, infos_s, prof_s, _ = timed(hs, "mixed", args.shared_steps, 1, profile=True)
            shared[key] = {"workload": f"{text} (n_v={wls.n_params:,}), 16,384 walkers x 4 samples",
                           "ms_per_step": round(ms_s, 3),
                           "sv_gbs": round(prof_s["pass_bytes"] / (prof_s["pass_ms"] * 1e-3) / 1e9, 1)
                           if prof_s and prof_s["pass_ms"] > 0 else None,
                           "cg_inner_iterations": float(np.mean([i["iterations"] for i in infos_s])),
                           "true_rel_residual": max(i["true_rel_residual"] for i in infos_s),
                           "converged": all(i["converged"] for i in infos_s)}
            hs.close()

    # ---- synthetic ab initio Hamiltonian (24 orbitals, 12+12 electrons, all
    # 276 pair correlators, two-electron integrals from 48 Cholesky vectors),
    # 8,192 walkers x 8 samples, mixed path: the SR step and, alone, the
    # sampling + local-energy pass (every single and double excitation of
    # each sample) ----------------------------------------------------------
    abinit = None
    if args.abinitio_steps > 0:
        wla = inputs.workload("abinitio24")
        ha = V.vmc_create(wla, walker_precision=V.VMC_FP32, keep_fp64_store=False, keep_lowp_store=True)
        V.vmc_set_params(ha, wla.C, wla.f)
        V.vmc_set_walkers(ha, wla.init_occ)
        sa = inputs.seed_sampling_for("abinitio24") + 7919 * rank
        V.vmc_sample(ha, wla.burn_in_sweeps, sa)
        ms_a, infos_a, prof_a, _ = timed(ha, "mixed", args.abinitio_steps, 1, profile=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        e0.record()
        for k in range(args.abinitio_steps):
            V.vmc_sample(ha, 0, sa + 100 + k)
        e1.record()
        barrier()
        ms_walk = e0.elapsed_time(e1) / args.abinitio_steps
        ns_orb, nu, nd = wla.n_sites, wla.n_up, wla.n_dn
        eu, ed = ns_orb - nu, ns_orb - nd
        n_dbl = (nu * (nu - 1) // 2) * (eu * (eu - 1) // 2) + (nd * (nd - 1) // 2) * (ed * (ed - 1) // 2) \
            + nu * nd * eu * ed
        n_sgl = nu * eu + nd * ed
        abinit = {"workload": f"synthetic ab initio, 24 orbitals, 12+12 electrons, 276 pair correlators + pfaffian "
                              f"(n_v={wla.n_params:,}), (pq|rs) from 48 Cholesky vectors, 8,192 walkers x 8 samples",
                  "ms_per_step": round(ms_a, 3),
                  "sample_and_local_energy_ms": round(ms_walk, 3),
                  "excitations_per_sample": {"single": n_sgl, "double": n_dbl},
                  "double_excitations_per_s": round(wla.n_samples * n_dbl / (ms_walk * 1e-3), 1),
                  "sv_gbs": round(prof_a["pass_bytes"] / (prof_a["pass_ms"] * 1e-3) / 1e9, 1)
                  if prof_a and prof_a["pass_ms"] > 0 else None,
                  "cg_inner_iterations": float(np.mean([i["iterations"] for i in infos_a])),
                  "true_rel_residual": max(i["true_rel_residual"] for i in infos_a),
                  "converged": all(i["converged"] for i in infos_a)}
        # accelerated linear method (Sec. II.B) on the same samples: the Eq. 10
        # product (H x, S x) through the Eq. 9 factors, and a bounded Davidson
        # solve of the shifted Eq. 8
        lm = None
        if args.lm_iters > 0:
            xl = torch.from_numpy(np.random.default_rng(0).standard_normal(wla.n_params + 1)).cuda()
            V.lm_apply(ha, xl, V.VMC_STORE_FP32)
            barrier()
            e0.record()
            for _ in range(3):
                V.lm_apply(ha, xl, V.VMC_STORE_FP32)
            e1.record()
            barrier()
            ms_lm = e0.elapsed_time(e1) / 3
            t0 = time.perf_counter()
            _, linfo = V.lm_solve(ha, 1.0, 1e-2, 1e-6, max_iter=args.lm_iters, max_sub=32,
                                  store=V.VMC_STORE_FP32, allow_not_converged=True)
            barrier()
            lm = {"product_ms": round(ms_lm, 3),
                  "products_per_s": round(1e3 / ms_lm, 2),
                  "davidson_s": round(time.perf_counter() - t0, 3),
                  "davidson": {k: (round(v, 6) if isinstance(v, float) else v) for k, v in linfo.items()},
                  "shifts": {"H": 1.0, "S": 1e-2}, "store": "fp32 (FP64 sums)"}
        abinit["linear_method"] = lm
        ha.close()

    # ---- plain FP64 path ------------------------------------------------------
    peak, peak_kind = peaks()
    fp64 = None
    if not args.no_fp64:
        hf = make("fp64")
        ms64, infos64, prof64, clocks64 = timed(hf, "fp64", max(1, args.fp64_steps), 1, profile=True)
        V.vmc_profile(hf, True)
        for _ in range(3):
            V.sr_apply_S(hf, torch.ones(wl.n_params, dtype=torch.float64, device="cuda"), shift, V.VMC_STORE_FP64)
        p64 = V.vmc_profile_read(hf, V.VMC_STORE_FP64)
        V.vmc_profile(hf, False)
        ms_p64 = p64["pass_ms"] / max(1, p64["pass_launches"])
        # FP64 FMAs of one product: t_s and t_s O_s over n_corr + P entries per sample
        fma = 2.0 * wl.n_samples * (wl.n_corr + wl.n_pf_block)
        fp64 = {"ms_per_step": round(ms64, 3),
                "cg_iterations": float(np.mean([i["iterations"] for i in infos64])),
                "true_rel_residual": max(i["true_rel_residual"] for i in infos64),
                "converged": all(i["converged"] for i in infos64),
                "roofline": {"bound": "alu", "kernel": "k_sr_main<double,double,1> (FP64 store, FP64 FMA)",
                             "product_ms": round(ms_p64, 4),
                             "achieved": round(2 * fma / (ms_p64 * 1e-3) / 1e12, 3), "unit": "TFLOP/s",
                             "peak": FP64_PEAK_TFLOPS, "peak_kind": "nominal FP64 rate of the GB300",
                             "frac": round(2 * fma / (ms_p64 * 1e-3) / 1e12 / FP64_PEAK_TFLOPS, 4),
                             "hbm_gbs": round(p64["pass_bytes"] / max(1, p64["pass_launches"]) / (ms_p64 * 1e-3) / 1e9, 1),
                             "hbm_frac": round(p64["pass_bytes"] / max(1, p64["pass_launches"])
                                               / (ms_p64 * 1e-3) / 1e9 / peak, 4)}}
        hf.close()

    # ---- lattices of uneven size in one launch: the 8x8 / 2x2-plaquette
    # workload (16,384 walkers x 8, N = 56) with the 4x4 pair workload (64 x 64,
    # N = 16): sampling and the FP32-store product, batched against separate --
    batch = None
    if args.batch_steps > 0:
        wb4, wb1 = inputs.workload("hubbard8x8_2x2"), inputs.workload("hubbard4x4_pair")
        hb = [make("mixed", wb4), make("mixed", wb1)]
        reps = args.batch_steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def clock(fn):
            fn(0)
            barrier()
            e0.record()
            for k in range(reps):
                fn(1 + k)
            e1.record()
            barrier()
            return e0.elapsed_time(e1) / reps

        ms_sep = clock(lambda k: [V.vmc_sample(h, 0, seed + 50 + 2 * k + j) for j, h in enumerate(hb)])
        ms_bat = clock(lambda k: V.vmc_sample_batch(hb, 0, [seed + 50 + 2 * k, seed + 51 + 2 * k]))
        for h in hb:
            V.sr_gradient(h, V.VMC_STORE_FP32, stats=False)
        vs = [torch.ones(w.n_params, dtype=torch.float64, device="cuda") for w in (wb4, wb1)]
        ms_psep = clock(lambda k: [V.sr_apply_S(h, v, shift, V.VMC_STORE_FP32) for h, v in zip(hb, vs)])
        ms_pbat = clock(lambda k: V.sr_apply_S_batch(hb, vs, shift, V.VMC_STORE_FP32))
        batch = {"workloads": ["hubbard8x8_2x2 (16,384 walkers x 8, N = 56)", "hubbard4x4_pair (64 x 64, N = 16)"],
                 "sample_separate_ms": round(ms_sep, 3), "sample_batched_ms": round(ms_bat, 3),
                 "fp32_store_product_separate_ms": round(ms_psep, 3),
                 "fp32_store_product_batched_ms": round(ms_pbat, 3)}
        for h in hb:
            h.close()

    # ---- the other workloads: the same SR step (mixed and FP64) ---------------
    configs = None
    if args.config_steps > 0:
        configs = {}
        for name in ("hubbard4x4_pair", "hubbard4x4_2x2", "hubbard8x8_2x2"):
            wlc = inputs.workload(name)
            row = {"n_params": wlc.n_params, "n_samples": wlc.n_samples}
            for path in ("mixed", "fp64"):
                hc = make(path, wlc)
                if path == "mixed":
                    row["autotune"] = tune(hc, f"{name}:{wlc.n_samples}")
                ms_c, infos_c, pc, _ = timed(hc, path, args.config_steps, 1, profile=True)
                gbs = pc["pass_bytes"] / (pc["pass_ms"] * 1e-3) / 1e9 if pc and pc["pass_ms"] > 0 else None
                row[path] = {"ms_per_step": round(ms_c, 3),
                             "cg_iterations": float(np.mean([i["iterations"] for i in infos_c])),
                             "true_rel_residual": max(i["true_rel_residual"] for i in infos_c),
                             "converged": all(i["converged"] for i in infos_c),
                             "sv_gbs": round(gbs, 1) if gbs else None,
                             "sv_frac_of_hbm": round(gbs / peak, 4) if gbs else None}
                hc.close()
            configs[name] = row

    ach = prof["pass_bytes"] / (prof["pass_ms"] * 1e-3) / 1e9 if prof and prof["pass_ms"] > 0 else None
    path1 = tuning["path"]
    per_launch_bytes = prof["pass_bytes"] / max(1, prof["pass_launches"]) if prof else None
    res = {
        "metric": METRIC,
        "value": round(ms / 1e3, 6),
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "precision": {"walkers": "f32 (inverse rebuilt from scratch each step)", "O_stream": "bf16",
                      "stream_accumulate": "f32", "scalars_and_outer_residual": "f64 over the f32 store",
                      "fp64_refresh_leg": "see refresh64: stored samples from FP64, residual vs the FP64 operator"},
        "autotune": tuning,
        "refresh64": refresh,
        "configs": configs,
        "batched_lattices": batch,
        "data": "synthetic (seeded random CPS amplitudes 1+N(0,0.01^2), pairing N(0,0.1^2), random sector starts)",
        "config": {"workload": WORKLOAD, "n_params": wl.n_params, "n_samples": wl.n_samples,
                   "shift": shift, "tol": tol, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (BF16 O store 214 MB, FP32 store 428 MB > 129 MB L2)"},
        "cg": {"inner_iterations": float(np.mean([i["iterations"] for i in infos])),
               "outer_steps": float(np.mean([i["refinements"] for i in infos])),
               "true_rel_residual": max(i["true_rel_residual"] for i in infos),
               "converged": all(i["converged"] for i in infos)},
        "sv_gbs": round(ach, 1) if ach else None,
        "fp64_path": fp64,
        "block_cg": block,
        "shared_correlators": shared,
        "abinitio": abinit,
        "speedup_vs_fp64_path": round(fp64["ms_per_step"] / ms, 3) if fp64 else None,
        "roofline": {"bound": "hbm", "kernel": PASS_KERNELS.get(path1, path1),
                     "achieved": round(ach, 1) if ach else None, "peak": peak, "unit": "GB/s",
                     "frac": round(ach / peak, 4) if ach else None, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": per_launch_bytes,
                     "launches": prof["pass_launches"] if prof else None,
                     "traffic": PASS_DRAM_BYTES.get(path1)},
        "e2e": {"value": round(float(np.median(e2e_ms)) / 1e3, 6), "unit": "s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(prof["launches_all"]) if prof else None,
        "clocks": clocks,
    }
    hm.close()
    return res, infos


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_step(n_walkers: int, spw: int, seed: int, cg_iters_full: float, name: str = "hubbard8x8_2x3",
                full: int = 65536):
    """The oracle's SR iteration on a bounded sample of a workload:
    n_walkers chains x spw samples (one sweep each, chains started from the
    thermalised-free seeded starts after one sweep), E_L and dense O, the
    gradient and one Eq. 7 product timed; scaled to the workload's `full`
    samples and its FP64 CG iteration count."""
    import oracle
    from paper_1108_0900_gb300 import inputs

    wl = inputs.workload(name, n_walkers=n_walkers, samples_per_walker=spw)
    P = oracle.Problem(wl)
    occ = wl.init_occ.copy()
    step = np.zeros(n_walkers, np.uint64)
    t0 = time.perf_counter()
    smp, _, _ = P.sample(occ, step, seed, 0, spw)
    t1 = time.perf_counter()
    E, O = P.measure(smp)
    t2 = time.perf_counter()
    g, _ = oracle.gradient(O, E)
    t3 = time.perf_counter()
    v = np.random.default_rng(0).standard_normal(wl.n_params)
    Ob = oracle.mean_O(O)
    n_prod = 5
    for _ in range(n_prod):
        oracle.apply_S(O, v, wl.shift, Obar=Ob)
    t4 = t3 + (time.perf_counter() - t3) / n_prod
    n = len(smp)
    per_sample = (t1 - t0 + t2 - t1 + t3 - t2) / n
    sv_per_sample = (t4 - t3) / n
    est = per_sample * full + sv_per_sample * full * cg_iters_full
    return est, {"sample_s": t1 - t0, "measure_s": t2 - t1, "gradient_s": t3 - t2, "apply_S_s": t4 - t3,
                 "n_samples": n}


def cpu_baseline(cg_iters_full: float, n_walkers=128, spw=2, configs=None):
    """The oracle on bounded samples: the headline workload on all host cores
    and on one core, and (configs: {name: (samples of the full workload, FP64
    CG iterations)}) the other workloads on all cores."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    est, parts = oracle_step(n_walkers, spw, 2005, cg_iters_full)
    # the same on one core, on a quarter of the sample
    oracle.set_threads(1)
    est1, parts1 = oracle_step(max(8, n_walkers // 4), spw, 2006, cg_iters_full)
    oracle.set_threads(cores)
    per_config = {}
    for name, (full, iters) in (configs or {}).items():
        nw = 16 if name.startswith("abinitio") else 64
        e, pc = oracle_step(nw, 1, 2007, iters, name=name, full=full)
        per_config[name] = {"value": round(e, 3), "unit": "s", "cores": int(cores), "n_samples": pc["n_samples"],
                            "full_samples": full, "cg_products": iters}
    return {"value": round(est, 3), "unit": "s", "cores": int(cores),
            "kind": "oracle",
            "sample": (f"{parts['n_samples']} samples ({n_walkers} walkers x {spw}) of the same workload: "
                       f"sampling + E_L + dense O + gradient timed and scaled x{65536 / parts['n_samples']:.0f}, "
                       f"Eq. 7 products (mean of 5) scaled to 65,536 samples x {cg_iters_full:.0f} CG products "
                       f"(the GPU FP64 path's iteration count)"),
            "nproc": int(cores),
            "one_core": {"value": round(est1, 3), "unit": "s", "cores": 1, "n_samples": parts1["n_samples"]},
            "configs": per_config,
            "parts": {k: round(v, 4) if isinstance(v, float) else v for k, v in parts.items()}}


def run_reference(args):
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    iters = args.ref_cg_iters
    vals = []
    for k in range(args.warmup + args.steps):
        est, parts = oracle_step(32, 2, 3000 + k, iters)
        if k >= args.warmup:
            vals.append(est)
    v = float(np.mean(vals))
    cb = {"value": round(v, 3), "unit": "s", "cores": int(os.environ["OMP_NUM_THREADS"]), "kind": "oracle",
          "sample": (f"each step: 64 samples (32 walkers x 2) of the same workload through the FP64 CPU oracle, "
                     f"scaled to 65,536 samples and {iters} CG products")}
    return {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD}, "cpu_baseline": cb,
            "e2e": {"value": round(v, 3), "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_sv_only(args):
    """S product timing on the same workload: the O store filled from seeded
    sector configurations (vmc_measure, FP32 walkers), then `--sv-only`
    passes per store kind, each timed on the device by the library's events."""
    import torch
    from paper_1108_0900_gb300 import inputs
    from paper_1108_0900_gb300 import vmcsr as V

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    wl = inputs.workload("hubbard8x8_2x3")
    h = V.vmc_create(wl, walker_precision=V.VMC_FP32, keep_fp64_store=True, keep_lowp_store=True)
    V.vmc_set_params(h, wl.C, wl.f)
    cfgs = inputs.draw_configs(np.random.default_rng(555), wl.n_samples, wl.n_sites, wl.n_up, wl.n_dn)
    V.vmc_measure(h, cfgs)
    peak, peak_kind = peaks()
    rng = np.random.default_rng(1)
    v1 = torch.from_numpy(rng.standard_normal(wl.n_params)).cuda()
    v4 = torch.from_numpy(rng.standard_normal((4, wl.n_params))).cuda()
    out = {}
    for name, store, path, v in (("bf16_sorted", V.VMC_STORE_BF16, V.VMC_PATH_SORTED, v1),
                                 ("bf16_fused", V.VMC_STORE_BF16, V.VMC_PATH_FUSED, v1),
                                 ("fp32_f32acc", V.VMC_STORE_FP32_F32ACC, V.VMC_PATH_AUTO, v1),
                                 ("fp32_f64acc", V.VMC_STORE_FP32, V.VMC_PATH_AUTO, v1),
                                 ("fp64", V.VMC_STORE_FP64, V.VMC_PATH_AUTO, v1),
                                 ("bf16_sorted_4_vectors", V.VMC_STORE_BF16, V.VMC_PATH_SORTED, v4)):
        V.vmc_set_product_path(h, path)
        for _ in range(2):
            V.sr_apply_S(h, v, wl.shift, store)
        torch.cuda.synchronize()
        V.vmc_profile(h, True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.sv_only):
            V.sr_apply_S(h, v, wl.shift, store)
        e1.record()
        torch.cuda.synchronize()
        pr = V.vmc_profile_read(h, store)
        V.vmc_profile(h, False)
        kms = pr["pass_ms"] / max(1, pr["pass_launches"])
        gbs = pr["pass_bytes"] / max(1, pr["pass_launches"]) / (kms * 1e-3) / 1e9
        out[name] = {"apply_S_ms": round(e0.elapsed_time(e1) / args.sv_only, 4), "stream_kernel_ms": round(kms, 4),
                     "stream_kernel_gbs": round(gbs, 1), "frac_of_hbm": round(gbs / peak, 4),
                     "algorithmic_bytes": pr["pass_bytes"] / max(1, pr["pass_launches"])}
    h.close()
    return {"metric": "S·v GB/s", "workload": WORKLOAD, "peak_gbs": peak, "peak_kind": peak_kind,
            "passes": args.sv_only, "stores": out}


def run_sample_only(args):
    """vmc_sample timing (Metropolis sweeps, local energies, derivative ratios)
    on a named workload with FP32 walkers: `--sample-only NAME`, `--sample-walkers`
    chains x the workload's samples per walker, `--steps` timed calls."""
    import torch
    from paper_1108_0900_gb300 import inputs
    from paper_1108_0900_gb300 import vmcsr as V

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    over = {"n_walkers": args.sample_walkers} if args.sample_walkers else {}
    wl = inputs.workload(args.sample_only, **over)
    h = V.vmc_create(wl, walker_precision=V.VMC_FP32, keep_fp64_store=False, keep_lowp_store=True)
    V.vmc_set_params(h, wl.C, wl.f)
    V.vmc_set_walkers(h, wl.init_occ)
    seed = inputs.seed_sampling_for(args.sample_only)
    V.vmc_sample(h, 2, seed)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        V.vmc_sample(h, 0, seed + 1 + k)
    e1.record()
    torch.cuda.synchronize()
    h.close()
    return {"workload": args.sample_only, "n_walkers": wl.n_walkers, "samples_per_walker": wl.samples_per_walker,
            "sample_ms": round(e0.elapsed_time(e1) / args.steps, 3), "calls": args.steps}


def run_lm_only(args):
    """Linear-method product timing on the 24-orbital ab initio workload:
    the stores filled from seeded sector configurations (vmc_measure, FP64
    walkers), then `--lm-only` Eq. 10 products per store, CUDA events on the
    launching stream."""
    import torch
    from paper_1108_0900_gb300 import inputs
    from paper_1108_0900_gb300 import vmcsr as V

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    wl = inputs.workload("abinitio24")
    h = V.vmc_create(wl, walker_precision=V.VMC_FP64, keep_fp64_store=True, keep_lowp_store=True)
    V.vmc_set_params(h, wl.C, wl.f)
    cfgs = inputs.draw_configs(np.random.default_rng(555), wl.n_samples, wl.n_sites, wl.n_up, wl.n_dn)
    V.vmc_measure(h, cfgs)
    x = torch.from_numpy(np.random.default_rng(2).standard_normal(wl.n_params + 1)).cuda()
    out = {}
    for name, store in (("fp32", V.VMC_STORE_FP32), ("fp64", V.VMC_STORE_FP64)):
        V.lm_apply(h, x, store)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.lm_only):
            V.lm_apply(h, x, store)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"product_ms": round(e0.elapsed_time(e1) / args.lm_only, 3)}
    h.close()
    return {"metric": "linear-method product ms", "workload": "synthetic ab initio, 24 orbitals, 12+12 electrons, "
            "276 pair correlators + pfaffian (n_v=5,544), 65,536 seeded sector configurations",
            "products": args.lm_only, "stores": out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--shared-steps", type=int, default=2,
                    help="SR steps timed on the shared-correlator 8x8 workload (0: skip)")
    ap.add_argument("--block-steps", type=int, default=2,
                    help="SR steps timed with the block-CG inner solve (0: skip)")
    ap.add_argument("--abinitio-steps", type=int, default=2,
                    help="SR steps timed on the 24-orbital ab initio workload (0: skip)")
    ap.add_argument("--lm-iters", type=int, default=60,
                    help="Davidson steps of the linear-method leg on the ab initio workload (0: skip)")
    ap.add_argument("--refresh-steps", type=int, default=2,
                    help="steps of the FP64-refresh / MIXED64 leg (0 to skip)")
    ap.add_argument("--config-steps", type=int, default=2,
                    help="steps per path of the other workloads (0 to skip)")
    ap.add_argument("--batch-steps", type=int, default=3,
                    help="timed calls of the batched-lattice leg (0 to skip)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-cg-iters", type=float, default=350.0)
    ap.add_argument("--sv-only", type=int, default=0, help="time N S products per store kind and exit")
    ap.add_argument("--lm-only", type=int, default=0, help="time N linear-method products per store and exit")
    ap.add_argument("--sample-only", default="", help="time vmc_sample on the named workload and exit")
    ap.add_argument("--sample-walkers", type=int, default=0, help="walkers of --sample-only (0: the workload's)")
    args = ap.parse_args()
    if args.sample_only:
        print(json.dumps(run_sample_only(args)))
        return
    if args.sv_only:
        print(json.dumps(run_sv_only(args)))
        return
    if args.lm_only:
        print(json.dumps(run_lm_only(args)))
        return
    args.warmup = max(args.warmup, 1)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res, infos = run_gpu(args, rank, world, dist)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            iters = (res["fp64_path"] or {}).get("cg_iterations") or res["cg"]["inner_iterations"]
            others = {name: (row["n_samples"], row["fp64"]["cg_iterations"])
                      for name, row in (res.get("configs") or {}).items()}
            if res.get("abinitio"):   # no FP64 leg there: the mixed solve's inner count
                others["abinitio24"] = (65536, res["abinitio"]["cg_inner_iterations"])
            res["cpu_baseline"] = cpu_baseline(iters, configs=others)
        print(json.dumps(res))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
