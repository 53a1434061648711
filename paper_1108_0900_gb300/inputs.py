"""Seeded synthetic workloads for the CPS x pfaffian SR hot path.

This module only *describes* problems: lattice geometry and bond lists,
correlator site lists, parameter draws, initial walker configurations and
ab initio integrals.  It holds none of the method's arithmetic (no amplitudes,
no local energies, no derivative ratios, no S products); the CPU oracle and
the CUDA library each implement those on their own and both consume the
plain arrays produced here.

Conventions (fixed here because the paper states none of them):
  * spatial site of lattice point (x, y) is ``y * Lx + x``;
  * spin orbital index is ``sigma * n_sites + site`` (all up, then all down);
  * Hubbard bonds are (i, i + x) and (i, i + y) for every site with periodic
    wrap; on a lattice of extent 2 the wrapped bond repeats and is kept twice;
  * a 2x2 plaquette anchored at (x, y) lists its sites as
    (x, y), (x+1, y), (x, y+1), (x+1, y+1); a 2x3 plaquette lists
    (x+dx, y+dy) with dy = 0..2 outer and dx = 0..1 inner;
  * correlator parameters come first (correlator-major, local state inner),
    then the pairing amplitudes f_pq, p < q, in row-major upper-triangle order;
  * C = 1 + N(0, 0.01^2), f = N(0, 0.1^2) (the 0.01 and 0.1 of the workload
    descriptions are read as standard deviations).

The workloads mirror the shapes of the paper's examples (Section III: 4x4 and
8x8 periodic Hubbard lattices with pair / plaquette correlators, and a
24-orbital ab initio active space), with synthetic values because the paper's
optimised parameters and integrals are not available.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

HUBBARD = 0
ABINITIO = 1


@dataclass
class Workload:
    name: str
    n_sites: int
    n_up: int
    n_dn: int
    ham: int                               # HUBBARD or ABINITIO
    corr_sites: List[np.ndarray]           # site list per correlator
    C: np.ndarray                          # float64 [n_corr_params]
    f: np.ndarray                          # float64 [M(M-1)/2]
    bonds: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    bond_t: np.ndarray = field(default_factory=lambda: np.zeros(0))
    U: float = 0.0
    h: Optional[np.ndarray] = None         # ab initio one-body [n_sites, n_sites]
    chol: Optional[np.ndarray] = None      # ab initio factors L[mu, p, q]
    n_walkers: int = 64
    samples_per_walker: int = 64
    burn_in_sweeps: int = 50
    shift: float = 1e-3
    tol: float = 1e-8
    seed_problem: int = 0
    seed_sampling: int = 0
    init_occ: Optional[np.ndarray] = None  # uint8 [n_walkers, N] ascending
    corr_class: Optional[np.ndarray] = None  # int32 [n_corr]: correlators of one class share parameters

    @property
    def M(self) -> int:
        return 2 * self.n_sites

    @property
    def N(self) -> int:
        return self.n_up + self.n_dn

    @property
    def n_corr(self) -> int:
        return len(self.corr_sites)

    @property
    def corr_ptr(self) -> np.ndarray:
        ptr = np.zeros(self.n_corr + 1, np.int32)
        ptr[1:] = np.cumsum([len(s) for s in self.corr_sites])
        return ptr

    @property
    def corr_flat(self) -> np.ndarray:
        if not self.corr_sites:
            return np.zeros(0, np.int32)
        return np.concatenate(self.corr_sites).astype(np.int32)

    @property
    def classes(self) -> np.ndarray:
        """Class of every correlator (each its own class unless shared)."""
        if self.corr_class is None:
            return np.arange(self.n_corr, dtype=np.int32)
        return np.asarray(self.corr_class, np.int32)

    @property
    def class_off(self) -> np.ndarray:
        """Parameter offset of every class block (classes in index order), plus the total."""
        cl = self.classes
        n_class = int(cl.max()) + 1 if len(cl) else 0
        dim = np.zeros(n_class, np.int64)
        for c, q in enumerate(cl):
            dim[q] = 4 ** len(self.corr_sites[c])
        return np.concatenate([[0], np.cumsum(dim)]).astype(np.int64)

    @property
    def corr_param_off(self) -> np.ndarray:
        """Parameter index of state 0 of every correlator."""
        return self.class_off[self.classes]

    @property
    def n_corr_params(self) -> int:
        return int(self.class_off[-1])

    @property
    def n_pf_block(self) -> int:
        """Stored pairing derivatives per sample: pairs of occupied orbitals."""
        return self.n_up * (self.n_up - 1) // 2 + self.n_dn * (self.n_dn - 1) // 2 + self.n_up * self.n_dn

    @property
    def n_pf_params(self) -> int:
        return self.M * (self.M - 1) // 2

    @property
    def n_params(self) -> int:
        return self.n_corr_params + self.n_pf_params

    @property
    def n_samples(self) -> int:
        return self.n_walkers * self.samples_per_walker


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def site(x: int, y: int, Lx: int, Ly: int) -> int:
    return (y % Ly) * Lx + (x % Lx)


def square_bonds(Lx: int, Ly: int) -> np.ndarray:
    """(i, i+x) and (i, i+y) for every site, periodic; duplicates kept."""
    b = []
    for y in range(Ly):
        for x in range(Lx):
            i = site(x, y, Lx, Ly)
            b.append((i, site(x + 1, y, Lx, Ly)))
            b.append((i, site(x, y + 1, Lx, Ly)))
    return np.asarray(b, np.int32)


def bond_correlators(Lx: int, Ly: int) -> List[np.ndarray]:
    return [np.asarray(p, np.int32) for p in square_bonds(Lx, Ly)]


def plaquette_correlators(Lx: int, Ly: int, px: int, py: int) -> List[np.ndarray]:
    out = []
    for y in range(Ly):
        for x in range(Lx):
            s = [site(x + dx, y + dy, Lx, Ly) for dy in range(py) for dx in range(px)]
            out.append(np.asarray(s, np.int32))
    return out


def all_pair_correlators(n: int) -> List[np.ndarray]:
    return [np.asarray((i, j), np.int32) for i in range(n) for j in range(i + 1, n)]


# --------------------------------------------------------------------------
# draws
# --------------------------------------------------------------------------

def translation_classes(corr: str, n_corr: int, Lx: int = 1) -> np.ndarray:
    """Translation classes of the generated correlators: bond correlators
    alternate x and y bonds (two classes); 3x3 plaquettes form one class per
    sublattice of their anchor site (the two 3x3 correlators of the paper's
    4x4 study, Sec. III.A); other plaquettes of one shape form one class."""
    if corr == "pair":
        return (np.arange(n_corr) % 2).astype(np.int32)
    if corr == "3x3":
        a = np.arange(n_corr)
        return ((a % Lx + a // Lx) % 2).astype(np.int32)
    return np.zeros(n_corr, np.int32)


def draw_params(rng: np.random.Generator, corr_sites, M: int, corr_class=None):
    if corr_class is None:
        n_corr_params = int(sum(4 ** len(s) for s in corr_sites))
    else:
        dims = {}
        for c, q in enumerate(corr_class):
            dims[int(q)] = 4 ** len(corr_sites[c])
        n_corr_params = int(sum(dims.values()))
    C = 1.0 + 0.01 * rng.standard_normal(n_corr_params)
    f = 0.1 * rng.standard_normal(M * (M - 1) // 2)
    return C, f


def draw_configs(rng: np.random.Generator, n_walkers: int, n_sites: int,
                 n_up: int, n_dn: int) -> np.ndarray:
    """Uniform random sector-valid configurations, ascending occupied lists."""
    out = np.empty((n_walkers, n_up + n_dn), np.uint8)
    for w in range(n_walkers):
        up = np.sort(rng.choice(n_sites, n_up, replace=False))
        dn = np.sort(rng.choice(n_sites, n_dn, replace=False)) + n_sites
        out[w] = np.concatenate([up, dn])
    return out


def draw_abinitio(rng: np.random.Generator, n: int, n_chol: int):
    idx = np.arange(n)
    decay = np.exp(-np.abs(idx[:, None] - idx[None, :]) / 4.0)
    r = rng.standard_normal((n, n))
    h = np.triu(r) + np.triu(r, 1).T
    h = h * decay
    L = rng.standard_normal((n_chol, n, n))
    L = 0.5 * (L + L.transpose(0, 2, 1)) * np.sqrt(2.0)
    L /= np.sqrt(n_chol)
    return h, L


# --------------------------------------------------------------------------
# named workloads (shapes follow the paper's Section III examples)
# --------------------------------------------------------------------------

def hubbard(name, Lx, Ly, n_up, n_dn, corr, U=4.0, t=1.0, seed=0,
            n_walkers=64, samples_per_walker=64, burn_in_sweeps=50,
            shift=1e-3, tol=1e-8, seed_sampling=None, shared=False) -> Workload:
    rng = np.random.default_rng(seed)
    n_sites = Lx * Ly
    if corr == "pair":
        cs = bond_correlators(Lx, Ly)
    elif corr == "2x2":
        cs = plaquette_correlators(Lx, Ly, 2, 2)
    elif corr == "2x3":
        cs = plaquette_correlators(Lx, Ly, 2, 3)
    elif corr == "3x3":
        cs = plaquette_correlators(Lx, Ly, 3, 3)
    elif corr == "none":
        cs = []
    else:
        raise ValueError(corr)
    cls = translation_classes(corr, len(cs), Lx) if shared and cs else None
    C, f = draw_params(rng, cs, 2 * n_sites, cls)
    bonds = square_bonds(Lx, Ly)
    init = draw_configs(rng, n_walkers, n_sites, n_up, n_dn)
    return Workload(name=name, n_sites=n_sites, n_up=n_up, n_dn=n_dn, ham=HUBBARD,
                    corr_sites=cs, C=C, f=f, bonds=bonds,
                    bond_t=np.full(len(bonds), t), U=U, n_walkers=n_walkers,
                    samples_per_walker=samples_per_walker,
                    burn_in_sweeps=burn_in_sweeps, shift=shift, tol=tol,
                    seed_problem=seed,
                    seed_sampling=seed + 1000 if seed_sampling is None else seed_sampling,
                    init_occ=init, corr_class=cls)


def abinitio(name, n_orb, n_up, n_dn, n_chol=48, seed=0, n_walkers=64,
             samples_per_walker=8, burn_in_sweeps=50, shift=1e-3, tol=1e-6,
             seed_sampling=None) -> Workload:
    rng = np.random.default_rng(seed)
    cs = all_pair_correlators(n_orb)
    C, f = draw_params(rng, cs, 2 * n_orb)
    h, L = draw_abinitio(rng, n_orb, n_chol)
    init = draw_configs(rng, n_walkers, n_orb, n_up, n_dn)
    return Workload(name=name, n_sites=n_orb, n_up=n_up, n_dn=n_dn, ham=ABINITIO,
                    corr_sites=cs, C=C, f=f, h=h, chol=L, n_walkers=n_walkers,
                    samples_per_walker=samples_per_walker,
                    burn_in_sweeps=burn_in_sweeps, shift=shift, tol=tol,
                    seed_problem=seed,
                    seed_sampling=seed + 1000 if seed_sampling is None else seed_sampling,
                    init_occ=init)


_WORKLOADS = {
    # name: (constructor, default sizes, problem seed, sampling seed)
    "hubbard4x4_pair": (lambda **kw: hubbard("hubbard4x4_pair", 4, 4, 8, 8, "pair", **kw),
                        dict(n_walkers=64, samples_per_walker=64, shift=1e-3, tol=1e-8), 1001, 2001),
    "hubbard4x4_2x2": (lambda **kw: hubbard("hubbard4x4_2x2", 4, 4, 8, 8, "2x2", **kw),
                       dict(n_walkers=4096, samples_per_walker=16, tol=1e-6), 1002, 2002),
    "abinitio24": (lambda **kw: abinitio("abinitio24", 24, 12, 12, **kw),
                   dict(n_walkers=8192, samples_per_walker=8, tol=1e-6), 1003, 2003),
    "hubbard8x8_2x2": (lambda **kw: hubbard("hubbard8x8_2x2", 8, 8, 28, 28, "2x2", **kw),
                       dict(n_walkers=16384, samples_per_walker=8, tol=1e-6), 1004, 2004),
    "hubbard8x8_2x3": (lambda **kw: hubbard("hubbard8x8_2x3", 8, 8, 28, 28, "2x3", **kw),
                       dict(n_walkers=16384, samples_per_walker=4, tol=1e-6), 1005, 2005),
}
WORKLOAD_NAMES = tuple(_WORKLOADS)


def workload(name: str, **over) -> Workload:
    """One of the five synthetic workloads of the hot path, by name:
    hubbard4x4_pair (4x4 Hubbard, 8+8 electrons, pair correlators, 4,096
    samples, FP64 checks), hubbard4x4_2x2 (2x2 plaquettes, 65,536 samples),
    abinitio24 (24 orbitals, 12+12 electrons, all pair correlators, 65,536
    samples), hubbard8x8_2x2 (8x8, 28+28 electrons, 2x2 plaquettes, 131,072
    samples) and hubbard8x8_2x3 (8x8, 28+28 electrons, 2x3 plaquettes, 65,536
    samples).  Keyword arguments override the sizes."""
    ctor, kw, seed, _ = _WORKLOADS[name]
    kw = dict(kw)
    kw.update(over)
    return ctor(seed=seed, **kw)


def seed_sampling_for(name: str) -> int:
    """Seed of the Metropolis chains used with the named workload."""
    return _WORKLOADS[name][3]
