"""Sample-sharded SR across processes on CPU ranks (gloo, world size 2).

Each rank keeps half of the samples and only exchanges the sums the module
documents; the solve and x_0 must equal the single-process oracle solve over
all samples.  The rank-local sums come from the oracle's dense O rows (test
infrastructure); the library provides the same sums on the GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1108_0900_gb300 import inputs, shard


class DenseLocal:
    def __init__(self, O, E):
        self.O = torch.from_numpy(O)
        self.E = torch.from_numpy(E)

    def moments(self):
        return self.O.sum(0), (self.E[:, None] * self.O).sum(0), float(self.E.sum()), self.O.shape[0]

    def product(self, v):
        return self.O.T @ (self.O @ v)


def _problem():
    wl = inputs.hubbard("sh", 3, 2, 2, 2, "pair", seed=71, n_walkers=16)
    P = oracle.Problem(wl)
    occ = wl.init_occ.copy()
    step = np.zeros(wl.n_walkers, np.uint64)
    smp, _, _ = P.sample(occ, step, 72, 5, 8)
    E, O = P.measure(smp)
    return wl, E, O


def _rank(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        wl, E, O = _problem()
        mine = np.arange(len(E)) % world == rank          # interleaved halves of the samples
        res = shard.sr_step(DenseLocal(O[mine], E[mine]), 0.05, 1e-3, 1e-10, 5000)
        np.save(os.path.join(out, f"y{rank}.npy"), res["y"].numpy())
        np.save(os.path.join(out, f"x0{rank}.npy"), np.array([res["x0"], res["E_mean"], res["n"]]))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_cpu_ranks_reproduce_the_single_process_solve(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    wl, E, O = _problem()
    g, Em = oracle.gradient(O, E)
    y_ref, it, res, ok = oracle.cg(O, g, 1e-3, 1e-10)
    assert ok
    alpha = np.zeros(wl.n_params)
    _, x0_ref = oracle.sr_update(alpha, y_ref, 0.05, Em, O.mean(0))
    for r in range(world):
        y = np.load(tmp_path / f"y{r}.npy")
        x0, Er, n = np.load(tmp_path / f"x0{r}.npy")
        assert n == len(E)
        assert Er == pytest.approx(Em, rel=1e-13)
        assert np.linalg.norm(y - y_ref) <= 1e-8 * np.linalg.norm(y_ref)
        assert x0 == pytest.approx(x0_ref, rel=1e-10)
    # every rank holds the same solution
    assert np.array_equal(np.load(tmp_path / "y0.npy"), np.load(tmp_path / "y1.npy"))


class OracleLMLocal:
    """Rank-local linear-method sample means from the oracle (Eq. 10 over the
    rank's own samples)."""

    def __init__(self, P, smp, factors):
        self.P, self.smp, self.factors = P, smp, factors

    def lm_product(self, x):
        Hx, Sx = self.P.lm_apply(self.smp, self.factors, x.numpy())
        return torch.from_numpy(Hx), torch.from_numpy(Sx), len(self.smp)


def _lm_problem():
    wl = inputs.hubbard("shl", 3, 2, 2, 2, "pair", seed=73, n_walkers=10)
    P = oracle.Problem(wl)
    occ = wl.init_occ.copy()
    step = np.zeros(wl.n_walkers, np.uint64)
    smp, _, _ = P.sample(occ, step, 74, 5, 3)
    x = np.random.default_rng(75).standard_normal(wl.n_params + 1)
    return wl, P, smp, x


def _lm_rank(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        wl, P, smp, x = _lm_problem()
        idx, cut = np.arange(len(smp)), len(smp) // 3
        mine = idx < cut if rank == 0 else idx >= cut      # uneven shares: 1/3 and 2/3
        Hx, Sx = shard.lm_apply(OracleLMLocal(P, smp[mine], oracle.lm_factors(wl)), torch.from_numpy(x))
        np.save(os.path.join(out, f"lmH{rank}.npy"), Hx.numpy())
        np.save(os.path.join(out, f"lmS{rank}.npy"), Sx.numpy())
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_reproduce_the_linear_method_product(tmp_path):
    """Ranks holding 1/3 and 2/3 of the samples, one all-reduce: the Eq. 10
    products equal the single-process ones over all samples."""
    world = 2
    mp.spawn(_lm_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    wl, P, smp, x = _lm_problem()
    H_ref, S_ref = P.lm_apply(smp, oracle.lm_factors(wl), x)
    for r in range(world):
        Hx = np.load(tmp_path / f"lmH{r}.npy")
        Sx = np.load(tmp_path / f"lmS{r}.npy")
        assert np.linalg.norm(Hx - H_ref) <= 1e-12 * np.linalg.norm(H_ref)
        assert np.linalg.norm(Sx - S_ref) <= 1e-12 * np.linalg.norm(S_ref)
