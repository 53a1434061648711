"""Sample-sharded SR over several processes (Sec. II.A: the samples, and the
stored derivative ratios, are distributed over processors).

Every rank holds its own walkers and O rows; only sums cross ranks:

* per SR step, one sum all-reduce of (sum O, sum E_L O, sum E_L, n_s):
  2 n_v + 2 numbers;
* per S product, one sum all-reduce of sum_s (O_s . v) O_s: n_v numbers;
* per linear-method product (Sec. II.B, Eq. 10: a sample mean like Eq. 7),
  one sum all-reduce of n_r (H x)_r, n_r (S x)_r and n_r: 2 n_v + 3 numbers.

Everything else (the CG vectors and scalars, x_0) is then the same on every
rank.  ``local`` supplies the rank-local sums:

* ``local.moments() -> (sumO, sumEO, sumE, n)`` (float64 tensors [n_v], floats)
* ``local.product(v) -> sum_s (O_s . v) O_s`` (float64 tensor [n_v])
* ``local.lm_product(x) -> ((H x)_r, (S x)_r, n_r)``, the rank's own sample
  means (float64 tensors [n_v + 1]) and its sample count

``LibraryLocal`` provides them from a library handle (``sr_local_moments`` /
``sr_local_product``).  ``reduce`` sums a tensor over the ranks in place;
the default is ``torch.distributed.all_reduce``.  This module is host logic;
the single-GPU solve is ``sr_cg_solve`` in the library.
"""
from __future__ import annotations

import math

import torch


def _dist_sum(t):
    import torch.distributed as dist
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def global_moments(local, reduce=_dist_sum):
    """Global Obar, g = <E_L O> - <E_L> Obar, <E_L> and N from one all-reduce."""
    sO, sEO, sE, n = local.moments()
    nv = sO.numel()
    buf = torch.cat([sO.reshape(-1), sEO.reshape(-1),
                     torch.tensor([float(sE), float(n)], dtype=torch.float64, device=sO.device)])
    reduce(buf)
    N = float(buf[2 * nv + 1])
    E = float(buf[2 * nv]) / N
    Obar = buf[:nv] / N
    g = buf[nv:2 * nv] / N - E * Obar
    return Obar, g, E, N


def apply_S(local, v, Obar, N, shift, reduce=_dist_sum):
    """(S + shift I) v = (1/N) sum_ranks sum_s (O_s . v) O_s - Obar (Obar . v) + shift v (Eq. 7)."""
    raw = local.product(v).clone()
    reduce(raw)
    return raw / N - Obar * torch.dot(Obar, v) + shift * v


def cg(local, g, Obar, N, shift, tol, max_iter, reduce=_dist_sum):
    """CG on (S + shift I) y = g with x_0 = 0; returns (y, iterations, true relative residual)."""
    y = torch.zeros_like(g)
    r = g.clone()
    p = r.clone()
    rr = float(torch.dot(r, r))
    gn = math.sqrt(rr)
    it = 0
    while it < max_iter and gn > 0 and math.sqrt(rr) > tol * gn:
        q = apply_S(local, p, Obar, N, shift, reduce)
        alpha = rr / float(torch.dot(p, q))
        y += alpha * p
        r -= alpha * q
        rr_new = float(torch.dot(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    res = g - apply_S(local, y, Obar, N, shift, reduce)
    return y, it, (float(torch.linalg.vector_norm(res)) / gn if gn > 0 else 0.0)


def sr_step(local, tau, shift, tol, max_iter, reduce=_dist_sum):
    """One sharded SR solve: global moments, CG, and x_0 = 1 - tau <E_L> + tau Obar . y.
    The parameter step is -tau y / x_0 on every rank."""
    Obar, g, E, N = global_moments(local, reduce)
    y, it, res = cg(local, g, Obar, N, shift, tol, max_iter, reduce)
    x0 = 1.0 - tau * E + tau * float(torch.dot(Obar, y))
    return dict(y=y, x0=x0, E_mean=E, n=N, g=g, Obar=Obar, iterations=it, true_rel_residual=res)


def lm_apply(local, x, reduce=_dist_sum):
    """Linear-method products (H x, S x) over every rank's samples: the
    rank means weighted by the ranks' sample counts, from one all-reduce."""
    Hx, Sx, n = local.lm_product(x)
    nv1 = Hx.numel()
    buf = torch.cat([Hx.reshape(-1) * n, Sx.reshape(-1) * n,
                     torch.tensor([float(n)], dtype=torch.float64, device=Hx.device)])
    reduce(buf)
    N = float(buf[2 * nv1])
    return buf[:nv1] / N, buf[nv1:2 * nv1] / N


class LibraryLocal:
    """Rank-local sums from a library handle over one O store."""

    def __init__(self, h, store=None):
        from . import vmcsr as V
        self.V = V
        self.h = h
        self.store = V.VMC_STORE_FP64 if store is None else store

    def moments(self):
        return self.V.sr_local_moments(self.h, self.store)

    def product(self, v):
        return self.V.sr_local_product(self.h, v, self.store)

    def lm_product(self, x):
        Hx, Sx = self.V.lm_apply(self.h, x, self.store)
        return Hx, Sx, self.V.vmc_num_samples(self.h)
