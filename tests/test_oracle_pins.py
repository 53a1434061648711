"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks the oracle against something it does not compute: published
known-answer vectors, closed forms, library routines, exact eigenstates,
structural invariants of Eq. 3 / Eq. 7 / Eq. 11, or brute force on tiny
Hilbert spaces.  None of these need a GPU.
"""
import copy
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1108_0900_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# random-number generator
# ---------------------------------------------------------------------------

def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# ---------------------------------------------------------------------------
# pfaffian and inverse (Eq. 11's amplitude)
# ---------------------------------------------------------------------------

def _antisym(rng, n):
    B = rng.standard_normal((n, n))
    return B - B.T


@pytest.mark.parametrize("n", [2, 4, 6, 8, 12, 16, 24, 56])
def test_pfaffian_squared_is_determinant(n):
    rng = np.random.default_rng(n)
    A = _antisym(rng, n) * (0.3 if n > 20 else 1.0)
    la, s = oracle.pfaffian_log(A)
    sd, ld = np.linalg.slogdet(A)
    assert sd > 0 and s != 0
    assert abs(2 * la - ld) < 1e-9 * max(1.0, abs(ld))


def test_pfaffian_two_by_two_and_block_diagonal():
    assert oracle.pfaffian([[0.0, 1.7], [-1.7, 0.0]]) == pytest.approx(1.7, rel=1e-15)
    rng = np.random.default_rng(3)
    A1, A2 = _antisym(rng, 4), _antisym(rng, 6)
    Z = np.zeros((10, 10))
    Z[:4, :4], Z[4:, 4:] = A1, A2
    assert oracle.pfaffian(Z) == pytest.approx(oracle.pfaffian(A1) * oracle.pfaffian(A2), rel=1e-12)
    # explicit 4x4 formula: a01 a23 - a02 a13 + a03 a12
    a = A1
    assert oracle.pfaffian(a) == pytest.approx(a[0, 1] * a[2, 3] - a[0, 2] * a[1, 3] + a[0, 3] * a[1, 2],
                                               rel=1e-12)


@pytest.mark.parametrize("n", [4, 10, 20])
def test_pfaffian_congruence(n):
    rng = np.random.default_rng(100 + n)
    A = _antisym(rng, n)
    B = rng.standard_normal((n, n))
    assert oracle.pfaffian(B @ A @ B.T) == pytest.approx(np.linalg.det(B) * oracle.pfaffian(A), rel=1e-9)


def test_pfaffian_row_swap_sign():
    rng = np.random.default_rng(9)
    A = _antisym(rng, 8)
    P = np.eye(8)[[1, 0, 2, 3, 4, 5, 6, 7]]
    assert oracle.pfaffian(P @ A @ P.T) == pytest.approx(-oracle.pfaffian(A), rel=1e-12)


def test_inverse_against_identity():
    rng = np.random.default_rng(5)
    for n in (2, 16, 56):
        A = _antisym(rng, n)
        X = oracle.inverse(A)
        assert np.abs(X @ A - np.eye(n)).max() < 1e-9


# ---------------------------------------------------------------------------
# parameter layout: the paper's printed counts (Sec. III.A and III.C)
# ---------------------------------------------------------------------------

def _open_plaquettes(L):
    return [np.array([y * L + x, y * L + x + 1, (y + 1) * L + x, (y + 1) * L + x + 1], np.int32)
            for y in range(L - 1) for x in range(L - 1)]


def _layout_count(n_sites, corr_sites):
    wl = inputs.Workload(name="count", n_sites=n_sites, n_up=1, n_dn=1, ham=inputs.HUBBARD,
                         corr_sites=corr_sites, C=np.ones(sum(4 ** len(s) for s in corr_sites)),
                         f=np.zeros(2 * n_sites * (2 * n_sites - 1) // 2))
    return oracle.Problem(wl).n_params(), wl.n_params


def test_paper_parameter_counts():
    golden = {}
    for l in open(os.path.join(GOLDEN, "param_counts.txt")):
        if l.strip() and l[0] != "#":
            name, count = l.split()[:2]
            golden[name] = int(count)
    # Sec. III.A: 4x4 lattice, two 3x3 correlators (one per sublattice)
    c33 = [np.arange(9, dtype=np.int32), np.arange(9, dtype=np.int32) + 1]
    assert _layout_count(16, c33) == (golden["hubbard4x4_two_3x3"],) * 2
    # Sec. III.C: 4x4 open lattice, all 2x2 plaquettes plus every pair not
    # already inside one plaquette
    plaq = _open_plaquettes(4)
    inside = {tuple(sorted(p)) for q in plaq for p in itertools.combinations(q.tolist(), 2)}
    pairs = [np.array(p, np.int32) for p in itertools.combinations(range(16), 2) if p not in inside]
    assert _layout_count(16, plaq + pairs) == (golden["hlattice4x4_2x2_pairs"],) * 2


def test_correlator_state_is_a_bijection():
    wl = inputs.hubbard("t", 2, 2, 2, 2, "2x2", seed=1, n_walkers=1)
    P = oracle.Problem(wl)
    occ_all, _ = P.enumerate()
    seen = {P.corr_state(o, 0) for o in occ_all}
    # the plaquette covers all four sites: every state with 2 up + 2 down
    # electrons is distinct and inside [0, 256)
    assert len(seen) == len(occ_all) and max(seen) < 256 and min(seen) >= 0


# ---------------------------------------------------------------------------
# local energy: exact eigenstates give zero-variance E_L
# ---------------------------------------------------------------------------

def _hopping_matrix(wl):
    T = np.zeros((wl.n_sites, wl.n_sites))
    for (i, j), t in zip(wl.bonds, wl.bond_t):
        T[i, j] -= t
        T[j, i] -= t
    return T


@pytest.mark.parametrize("Lx,Ly,nu", [(4, 4, 8), (3, 2, 3), (4, 4, 5)])
def test_free_fermion_limit(Lx, Ly, nu):
    """U = 0, all C = 1, f_{i up, j dn} = sum_k phi_k(i) phi_k(j): Psi is a
    product of two Slater determinants of hopping eigenorbitals, so every
    configuration has E_L = 2 * (sum of the nu lowest eigenvalues)."""
    wl = inputs.hubbard("u0", Lx, Ly, nu, nu, "pair", U=0.0, seed=7, n_walkers=16)
    wl.C[:] = 1.0
    ns, M = wl.n_sites, wl.M
    eps, phi = np.linalg.eigh(_hopping_matrix(wl))
    F = phi[:, :nu] @ phi[:, :nu].T
    f = np.zeros(M * (M - 1) // 2)
    for i in range(ns):
        for j in range(ns):
            p, q = i, ns + j
            f[p * M - p * (p + 1) // 2 + (q - p - 1)] = F[i, j]
    wl.f = f
    P = oracle.Problem(wl)
    # the free-fermion state has exact nodes: start from configurations
    # whose amplitude is well away from them
    cand = inputs.draw_configs(np.random.default_rng(8), 256, ns, nu, nu)
    la = np.array([P.log_psi(o)[0] if P.log_psi(o)[1] != 0 else -np.inf for o in cand])
    occ = np.ascontiguousarray(cand[la > la.max() - 8][:16])
    step = np.zeros(len(occ), np.uint64)
    samples, _, _ = P.sample(occ, step, 11, 5, 4)
    E, _ = P.measure(samples, want_O=False)
    assert np.allclose(E, 2 * eps[:nu].sum(), atol=1e-8)


def test_two_site_hubbard_exact_state():
    """One bond, one up + one down electron.  With one correlator covering
    both sites set to psi_exact / f, E_L is (U - sqrt(U^2 + 16 t^2)) / 2 on
    all four configurations (closed form of the 2x2 Hamiltonian)."""
    U, t = 4.0, 1.0
    E0 = (U - np.sqrt(U * U + 16 * t * t)) / 2
    # basis (up site, down site): 00, 01, 10, 11; symmetric ground state
    a = 1.0
    b = -2 * t * a / E0
    psi = {(0, 0): a, (0, 1): b, (1, 0): b, (1, 1): a}
    wl = inputs.Workload(name="2site", n_sites=2, n_up=1, n_dn=1, ham=inputs.HUBBARD,
                         corr_sites=[np.array([0, 1], np.int32)], C=np.ones(16),
                         f=np.array([0.3, 0.7, -0.4, 0.9, 0.5, 0.2]),
                         bonds=np.array([[0, 1]], np.int32), bond_t=np.array([t]), U=U)
    M = 4
    for (i, j), v in psi.items():
        p, q = i, 2 + j
        fpq = wl.f[p * M - p * (p + 1) // 2 + (q - p - 1)]
        idx = (1 if i == 0 else 0) + 2 * (1 if j == 0 else 0) + 4 * ((1 if i == 1 else 0) + 2 * (1 if j == 1 else 0))
        wl.C[idx] = v / fpq
    P = oracle.Problem(wl)
    for (i, j) in psi:
        occ = np.array([i, 2 + j], np.uint8)
        assert P.local_energy(occ) == pytest.approx(E0, abs=1e-12)
    assert E0 == pytest.approx(-0.8284271247461903, abs=1e-12)


# ---------------------------------------------------------------------------
# brute force on tiny Hilbert spaces (Jordan-Wigner matrices in numpy)
# ---------------------------------------------------------------------------

def _jw_ops(M):
    """a_p as sparse 2^M matrices; bit p of the basis index = occupation of
    orbital p.  With a+_p = (prod_{o<p} Z_o) sigma+_p, the state
    a+_{o1} ... a+_{oN}|0> with o1 < ... < oN is the bit string with sign +."""
    import scipy.sparse as sp
    D = 1 << M
    ops = []
    for p in range(M):
        rows, cols, vals = [], [], []
        for s in range(D):
            if s >> p & 1:
                rows.append(s ^ (1 << p))
                cols.append(s)
                vals.append((-1) ** bin(s & ((1 << p) - 1)).count("1"))
        ops.append(sp.csr_matrix((vals, (rows, cols)), shape=(D, D)))
    return ops


def _jw_hamiltonian(wl):
    M, n = wl.M, wl.n_sites
    a = _jw_ops(M)
    ad = [x.T.tocsr() for x in a]
    H = 0 * a[0]
    if wl.ham == inputs.HUBBARD:
        for (i, j), t in zip(wl.bonds, wl.bond_t):
            for s in range(2):
                x, y = s * n + i, s * n + j
                H = H - t * (ad[x] @ a[y] + ad[y] @ a[x])
        for i in range(n):
            H = H + wl.U * (ad[i] @ a[i]) @ (ad[n + i] @ a[n + i])
    else:
        eri = np.einsum("mpq,mrs->pqrs", wl.chol, wl.chol)
        for s in range(2):
            for p in range(n):
                for q in range(n):
                    H = H + wl.h[p, q] * (ad[s * n + p] @ a[s * n + q])
        for s1 in range(2):
            for s2 in range(2):
                for p, q, r, s in itertools.product(range(n), repeat=4):
                    H = H + 0.5 * eri[p, q, r, s] * (ad[s1 * n + p] @ ad[s2 * n + r] @ a[s2 * n + s] @ a[s1 * n + q])
    return H.toarray()


def _bits(occ):
    return sum(1 << int(o) for o in occ)


@pytest.mark.parametrize("kind", ["hubbard2x2", "hubbard3x2", "abinitio3_11", "abinitio3_22", "abinitio4_22"])
def test_hamiltonian_elements_and_energy_identity(kind):
    if kind == "hubbard2x2":
        wl = inputs.hubbard("t", 2, 2, 2, 2, "2x2", seed=3, n_walkers=1)
    elif kind == "hubbard3x2":
        wl = inputs.hubbard("t", 3, 2, 1, 1, "pair", seed=3, n_walkers=1)
    elif kind == "abinitio3_11":
        wl = inputs.abinitio("t", 3, 1, 1, n_chol=4, seed=4, n_walkers=1)
    elif kind == "abinitio3_22":
        wl = inputs.abinitio("t", 3, 2, 2, n_chol=4, seed=5, n_walkers=1)
    else:                                   # the 4-orbital toy: 36 configurations, 256-dim Fock space
        wl = inputs.abinitio("t", 4, 2, 2, n_chol=5, seed=6, n_walkers=1)
    P = oracle.Problem(wl)
    H = _jw_hamiltonian(wl)
    occ_all, w = P.enumerate()
    idx = [_bits(o) for o in occ_all]
    Hs = H[np.ix_(idx, idx)]
    Ho = np.array([[P.hamiltonian_element(a, b) for b in occ_all] for a in occ_all])
    assert np.abs(Hs - Ho).max() < 1e-12
    # sum_n |Psi_n|^2 E_L(n) / <Psi|Psi> = <Psi|H|Psi> / <Psi|Psi>
    psi = np.array([np.exp(l) * s for l, s in (P.log_psi(o) for o in occ_all)])
    E, _ = P.measure(occ_all, want_O=False)
    lhs = np.sum(w * E)
    rhs = psi @ Hs @ psi / (psi @ psi)
    assert lhs == pytest.approx(rhs, rel=1e-10, abs=1e-12)


def _closed_shell_pairing(M, phi_occ):
    """f_{i up, j dn} = sum_k phi_k(i) phi_k(j): with C = 1, Psi is the
    product of the up and down Slater determinants of the orbitals phi_k."""
    ns = M // 2
    F = phi_occ @ phi_occ.T
    f = np.zeros(M * (M - 1) // 2)
    for i in range(ns):
        for j in range(ns):
            p, q = i, ns + j
            f[p * M - p * (p + 1) // 2 + (q - p - 1)] = F[i, j]
    return f


def test_abinitio_eigenstates_at_24_orbitals():
    """Closed forms for the ab initio local energy at the full 24-orbital,
    12 + 12 electron size (every single and double excitation enumerated):
    (a) one-body H (no Cholesky vectors), Psi = determinants of the 12 lowest
        eigenvectors of h: E_L = 2 (sum of those eigenvalues) on every sample;
    (b) H = 1/2 sum (pq|rs) a+ a+ a a with one Cholesky vector K (so H =
        Khat^2 / 2 - Jhat / 2, J = K^2), Psi = determinants of the 12 lowest
        eigenvectors of K: an eigenstate, E_L = kappa^2 / 2 - sum lambda_k^2
        with kappa = 2 sum lambda_k, on every sample (this exercises the
        double excitations);
    (c) diagonal h and a diagonal Cholesky vector d: H is diagonal and E_L(n)
        = sum_P h_pp n_P + (sum_P d_p n_P)^2 / 2 - sum_P d_p^2 n_P / 2 for any
        Psi."""
    n, M = 24, 48
    wl = inputs.abinitio("a", n, 12, 12, n_chol=1, seed=77, n_walkers=3)
    wl.C = np.ones_like(wl.C)
    wl.chol = np.zeros((1, n, n))
    eps, phi = np.linalg.eigh(wl.h)
    wl.f = _closed_shell_pairing(M, phi[:, :12])
    P = oracle.Problem(wl)
    for o in wl.init_occ:
        assert P.local_energy(o) == pytest.approx(2 * eps[:12].sum(), rel=1e-12, abs=1e-12)

    wl = inputs.abinitio("b", n, 12, 12, n_chol=1, seed=79, n_walkers=3)
    A = np.random.default_rng(9).standard_normal((n, n))
    K = 0.1 * (A + A.T)
    wl.h = np.zeros((n, n))
    wl.chol = K[None].copy()
    wl.C = np.ones_like(wl.C)
    lam, phi = np.linalg.eigh(K)
    wl.f = _closed_shell_pairing(M, phi[:, :12])
    P = oracle.Problem(wl)
    kappa = 2 * lam[:12].sum()
    for o in wl.init_occ:
        assert P.local_energy(o) == pytest.approx(0.5 * kappa ** 2 - lam[:12] @ lam[:12], rel=1e-12)

    wl = inputs.abinitio("c", n, 12, 12, n_chol=1, seed=78, n_walkers=3)
    d = np.random.default_rng(5).standard_normal(n)
    hd = np.random.default_rng(6).standard_normal(n)
    wl.h = np.diag(hd)
    wl.chol = np.diag(d)[None]
    P = oracle.Problem(wl)
    dd, hh = np.concatenate([d, d]), np.concatenate([hd, hd])
    for o in wl.init_occ:
        nocc = np.zeros(M)
        nocc[o] = 1.0
        ref = hh @ nocc + 0.5 * (dd @ nocc) ** 2 - 0.5 * (dd ** 2) @ nocc
        assert P.local_energy(o) == pytest.approx(ref, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("no,nu,nd", [(3, 1, 1), (4, 2, 2), (5, 2, 2), (5, 3, 1)])
def test_abinitio_local_energy_restricted_strings(no, nu, nd):
    """The local energy used at scale applies only the operator strings that
    can connect n' to n; it must equal the one built from the unrestricted
    operator sum (itself pinned by the Jordan-Wigner brute force above)."""
    wl = inputs.abinitio("t", no, nu, nd, n_chol=5, seed=10 + no, n_walkers=6)
    P = oracle.Problem(wl)
    for o in wl.init_occ:
        assert P.local_energy(o) == pytest.approx(P.local_energy_bruteforce(o), rel=1e-12, abs=1e-12)


# ---------------------------------------------------------------------------
# derivative ratios (Eq. 3): finite differences and structural invariants
# ---------------------------------------------------------------------------

def _with_params(wl, C, f):
    import copy
    w2 = copy.copy(wl)
    w2.C, w2.f = C, f
    return oracle.Problem(w2)


def test_logderiv_matches_finite_differences():
    wl = inputs.hubbard("fd", 3, 2, 2, 2, "pair", seed=21, n_walkers=3)
    P = oracle.Problem(wl)
    ncp = wl.n_corr_params
    h = 1e-6
    for occ in wl.init_occ:
        O = P.logderiv(occ)
        fd = np.zeros_like(O)
        for k in range(wl.n_params):
            C1, f1 = wl.C.copy(), wl.f.copy()
            C2, f2 = wl.C.copy(), wl.f.copy()
            if k < ncp:
                C1[k] += h
                C2[k] -= h
            else:
                f1[k - ncp] += h
                f2[k - ncp] -= h
            lp = _with_params(wl, C1, f1).log_psi(occ)[0]
            lm = _with_params(wl, C2, f2).log_psi(occ)[0]
            fd[k] = (lp - lm) / (2 * h)
        assert np.abs(O - fd).max() <= 1e-6 * max(1.0, np.abs(O).max())


def test_shared_correlators_logderiv_finite_differences():
    """Translation-invariant correlators (one parameter block per class):
    O of a shared parameter is the sum over the correlators reading it, which
    central differences of ln|Psi| see directly."""
    for corr in ("pair", "2x2"):
        wl = inputs.hubbard("fds", 3, 2, 2, 2, corr, seed=23, n_walkers=2, shared=True)
        assert wl.corr_class is not None and wl.n_corr_params == len(set(wl.corr_class)) * 4 ** len(wl.corr_sites[0])
        P = oracle.Problem(wl)
        ncp = wl.n_corr_params
        h = 1e-6
        for occ in wl.init_occ:
            O = P.logderiv(occ)
            for k in range(ncp):
                C1, C2 = wl.C.copy(), wl.C.copy()
                C1[k] += h
                C2[k] -= h
                lp = _with_params(wl, C1, wl.f).log_psi(occ)[0]
                lm = _with_params(wl, C2, wl.f).log_psi(occ)[0]
                assert abs(O[k] - (lp - lm) / (2 * h)) <= 1e-6 * max(1.0, abs(O[k]))
            # the states the correlators occupy, counted with multiplicity
            cnt = np.zeros(ncp)
            for c in range(wl.n_corr):
                cnt[wl.corr_param_off[c] + P.corr_state(occ, c)] += 1
            assert np.allclose(O[:ncp] * wl.C, cnt, atol=1e-12)


def test_shared_correlator_null_vectors_and_paper_count():
    """O_s . C_q = (number of correlators of class q) for every sample, so
    S C_q = eps C_q; and the paper's 4x4 layout, a 3x3 correlator at every
    site shared within each sublattice, has 2 x 4^9 + 496 = 524,784 parameters."""
    wl = inputs.hubbard("nvs", 4, 4, 5, 5, "2x2", seed=33, n_walkers=8, shared=True)
    P = oracle.Problem(wl)
    occ = wl.init_occ.copy()
    step = np.zeros(wl.n_walkers, np.uint64)
    samples, _, _ = P.sample(occ, step, 79, 3, 5)
    E, O = P.measure(samples)
    v = np.zeros(wl.n_params)
    v[:wl.n_corr_params] = wl.C
    assert np.allclose(O @ v, wl.n_corr, atol=1e-10)
    Sv = oracle.apply_S(O, v, 1e-3)
    assert np.abs(Sv - 1e-3 * v).max() < 1e-9
    g, _ = oracle.gradient(O, E)
    assert abs(g @ v) < 1e-8
    golden = {l.split()[0]: int(l.split()[1]) for l in open(os.path.join(GOLDEN, "param_counts.txt"))
              if l.strip() and l[0] != "#"}
    c33 = inputs.plaquette_correlators(4, 4, 3, 3)
    cls = np.array([(x + y) % 2 for y in range(4) for x in range(4)], np.int32)
    wl33 = inputs.Workload(name="c", n_sites=16, n_up=1, n_dn=1, ham=inputs.HUBBARD, corr_sites=c33,
                           C=np.ones(2 * 4 ** 9), f=np.zeros(32 * 31 // 2), corr_class=cls)
    assert oracle.Problem(wl33).n_params() == wl33.n_params == golden["hubbard4x4_two_3x3"]


def test_homogeneity_null_vectors():
    """O_s . C_c = 1 for every correlator block c and O_s . f = N/2 (the
    pfaffian is homogeneous of degree N/2 in f), so S C_c = eps C_c,
    S f = eps f and g . C_c = g . f = 0."""
    wl = inputs.hubbard("nv", 4, 4, 5, 5, "2x2", seed=31, n_walkers=8)
    P = oracle.Problem(wl)
    occ = wl.init_occ.copy()
    step = np.zeros(wl.n_walkers, np.uint64)
    samples, _, _ = P.sample(occ, step, 77, 3, 5)
    E, O = P.measure(samples)
    ncp = wl.n_corr_params
    vf = np.zeros(wl.n_params)
    vf[ncp:] = wl.f
    assert np.allclose(O @ vf, wl.N / 2, atol=1e-9)
    g, _ = oracle.gradient(O, E)
    eps = 1e-3
    for c in (0, 5, 15):
        v = np.zeros(wl.n_params)
        v[c * 256:(c + 1) * 256] = wl.C[c * 256:(c + 1) * 256]
        assert np.allclose(O @ v, 1.0, atol=1e-12)
        Sv = oracle.apply_S(O, v, eps)
        assert np.abs(Sv - eps * v).max() < 1e-10
        assert abs(g @ v) < 1e-9
    Sf = oracle.apply_S(O, vf, eps)
    assert np.abs(Sf - eps * vf).max() < 1e-9
    assert abs(g @ vf) < 1e-8


# ---------------------------------------------------------------------------
# S products (Eq. 3-7) and the CG solve
# ---------------------------------------------------------------------------

def _small_samples(seed=41, nw=16, spw=8):
    wl = inputs.hubbard("s", 3, 2, 2, 2, "pair", seed=seed, n_walkers=nw)
    P = oracle.Problem(wl)
    occ = wl.init_occ.copy()
    step = np.zeros(nw, np.uint64)
    samples, _, _ = P.sample(occ, step, seed + 5, 5, spw)
    E, O = P.measure(samples)
    return wl, P, samples, E, O


def test_apply_S_equals_dense_covariance():
    wl, P, samples, E, O = _small_samples()
    n = O.shape[0]
    Ob = O.mean(0)
    S_np = O.T @ O / n - np.outer(Ob, Ob)
    S_or = oracle.dense_S(O)
    assert np.abs(S_np - S_or).max() < 1e-12 * max(1, np.abs(S_np).max())
    rng = np.random.default_rng(0)
    for eps in (0.0, 1e-3):
        v = rng.standard_normal(wl.n_params)
        ref = S_np @ v + eps * v
        out = oracle.apply_S(O, v, eps)
        assert np.linalg.norm(out - ref) <= 1e-12 * np.linalg.norm(ref)
    g, Em = oracle.gradient(O, E)
    assert Em == pytest.approx(E.mean(), rel=1e-14)
    g_np = (E[:, None] * O).mean(0) - E.mean() * Ob
    assert np.abs(g - g_np).max() < 1e-12 * max(1, np.abs(g_np).max())


@pytest.mark.parametrize("shared", [False, True])
def test_apply_S_compact_equals_dense_rows(shared):
    """Eq. 7 from compact rows (occupation, correlator states, the N(N-1)/2
    pairing values in the documented block order) equals Eq. 7 over the dense
    O rows of the same samples.  The compact rows are first shown to be the
    dense rows: scattered back to n_v entries they reproduce every entry of
    the oracle's O (each correlator at 1/C of its state, each pairing value
    at f_{occ[a] occ[b]}), so nothing is dropped or misplaced."""
    from pair_blocks import block_pairs
    if shared:
        wl = inputs.hubbard("cmp", 3, 2, 2, 2, "2x2", seed=31, n_walkers=8, shared=True)
    else:
        wl = inputs.hubbard("cmp", 3, 2, 2, 2, "pair", seed=32, n_walkers=8)
    P = oracle.Problem(wl)
    occ = wl.init_occ.copy()
    samples, _, _ = P.sample(occ, np.zeros(wl.n_walkers, np.uint64), 77, 4, 6)
    _, O = P.measure(samples)
    n, N, M, ncp = len(samples), wl.N, wl.M, wl.n_corr_params
    pairs = block_pairs(wl.n_up, wl.n_dn)
    cs = np.array([[P.corr_state(o, c) for c in range(wl.n_corr)] for o in samples], np.int64)
    p = samples[:, pairs[:, 0]].astype(np.int64)
    q = samples[:, pairs[:, 1]].astype(np.int64)
    pq = ncp + p * M - p * (p + 1) // 2 + (q - p - 1)
    pf = np.take_along_axis(O, pq, axis=1)
    dense = np.zeros_like(O)
    for s_ in range(n):
        for c in range(wl.n_corr):
            k = wl.corr_param_off[c] + cs[s_, c]
            dense[s_, k] += 1.0 / wl.C[k]
        dense[s_, pq[s_]] = pf[s_]
    assert np.abs(dense - O).max() <= 1e-15 * max(1.0, np.abs(O).max())
    rng = np.random.default_rng(3)
    V = rng.standard_normal((2, wl.n_params))
    for eps in (0.0, 1e-3):
        out, Obar = oracle.apply_S_compact(P, samples, cs, pairs, pf, V, eps)
        assert np.abs(Obar - O.mean(0)).max() <= 1e-14
        for j in range(2):
            ref = oracle.apply_S(O, V[j], eps)
            assert np.linalg.norm(out[j] - ref) <= 1e-12 * np.linalg.norm(ref)
    out1, _ = oracle.apply_S_compact(P, samples, cs, pairs, pf, V[1], 1e-3)
    assert np.linalg.norm(out1 - oracle.apply_S(O, V[1], 1e-3)) <= 1e-12 * np.linalg.norm(out1)


def test_cg_matches_direct_solve():
    wl, P, samples, E, O = _small_samples(seed=43, nw=32, spw=8)
    g, _ = oracle.gradient(O, E)
    eps = 1e-3
    x, it, res, ok = oracle.cg(O, g, eps, 1e-10)
    assert ok and res <= 1e-9
    n = O.shape[0]
    Ob = O.mean(0)
    A = O.T @ O / n - np.outer(Ob, Ob) + eps * np.eye(wl.n_params)
    xs = np.linalg.solve(A, g)
    assert np.linalg.norm(x - xs) <= 1e-7 * np.linalg.norm(xs)


def test_exact_enumeration_gradient_and_S():
    """Weighted sums over the whole sector give the exact <E>, g and S; a
    long sampled estimate agrees within its statistical error."""
    wl = inputs.hubbard("ex", 2, 2, 2, 2, "2x2", seed=51, n_walkers=128)
    P = oracle.Problem(wl)
    occ_all, w = P.enumerate()
    assert len(occ_all) == 36 and abs(w.sum() - 1) < 1e-12
    E_all, O_all = P.measure(occ_all)
    E_ex = w @ E_all
    Ob_ex = w @ O_all
    # sampled
    occ = wl.init_occ.copy()
    step = np.zeros(wl.n_walkers, np.uint64)
    samples, _, _ = P.sample(occ, step, 99, 20, 40)
    E_s, O_s = P.measure(samples)
    per_walker = E_s.reshape(wl.n_walkers, -1).mean(1)
    err = per_walker.std(ddof=1) / np.sqrt(wl.n_walkers)
    assert abs(E_s.mean() - E_ex) < 4 * err + 1e-12
    # exact S is the weighted covariance; its Eq. 7 product with any vector
    S_ex = (O_all * w[:, None]).T @ O_all - np.outer(Ob_ex, Ob_ex)
    assert np.allclose(S_ex, S_ex.T)
    assert np.linalg.eigvalsh(S_ex).min() > -1e-12


def test_sr_update_solves_the_full_projection():
    """Sec. II.A update: solving the whole Eq. 2 system (row 0 with O_0 = 1
    included, eps on the derivative block only) by a dense solve gives the
    same x_0 and new parameters as the eliminated covariance solve plus the
    x_0 formula of the oracle."""
    wl, P, samples, E, O = _small_samples(seed=47, nw=16, spw=8)
    n, nv = O.shape
    eps, tau = 1e-3, 0.05
    Ob = O.mean(0)
    Oa = np.hstack([np.ones((n, 1)), O])                      # O_0 = 1
    G = Oa.T @ Oa / n
    G[1:, 1:] += eps * np.eye(nv)
    b = Oa.mean(0) - tau * (E[:, None] * Oa).mean(0)          # <Psi^i|(1 - tau H)|Psi> / <Psi|Psi>
    xf = np.linalg.solve(G, b)
    alpha = np.concatenate([wl.C, wl.f])
    ref = alpha + xf[1:] / xf[0]
    g, Em = oracle.gradient(O, E)
    y = np.linalg.solve(O.T @ O / n - np.outer(Ob, Ob) + eps * np.eye(nv), g)
    out, x0 = oracle.sr_update(alpha, y, tau, Em, Ob)
    assert x0 == pytest.approx(xf[0], rel=1e-10)
    assert np.linalg.norm(out - ref) <= 1e-10 * np.linalg.norm(ref)
    # no step for tau = 0
    out0, x00 = oracle.sr_update(alpha, y, 0.0, Em, Ob)
    assert x00 == 1.0 and np.array_equal(out0, alpha)


def test_sr_update_lowers_the_exact_energy_at_first_order():
    """With exact (enumerated) E, g and S on a 2x2 lattice the update moves
    alpha by -tau y / x_0, y = (S + eps)^-1 g, and the exact energy changes by
    2 g . dalpha + O(tau^2) (g is half the energy gradient): it goes down."""
    wl = inputs.hubbard("ex", 2, 2, 2, 2, "2x2", seed=53, n_walkers=8)
    P = oracle.Problem(wl)
    occ_all, w = P.enumerate()
    E_all, O_all = P.measure(occ_all)
    E_ex = w @ E_all
    Ob = w @ O_all
    g = w @ (E_all[:, None] * O_all) - E_ex * Ob
    S = (O_all * w[:, None]).T @ O_all - np.outer(Ob, Ob)
    eps = 1e-3
    y = np.linalg.solve(S + eps * np.eye(len(g)), g)
    alpha = np.concatenate([wl.C, wl.f])
    nc = len(wl.C)

    def exact_energy(a):
        wl2 = copy.copy(wl)
        wl2.C, wl2.f = a[:nc].copy(), a[nc:].copy()
        P2 = oracle.Problem(wl2)
        o2, w2 = P2.enumerate()
        return w2 @ P2.measure(o2)[0]

    slopes = []
    for tau in (1e-3, 1e-4):
        a2, x0 = oracle.sr_update(alpha, y, tau, E_ex, Ob)
        dE = exact_energy(a2) - E_ex
        assert dE < 0
        slopes.append(dE / tau)
        assert dE == pytest.approx(2 * g @ (a2 - alpha), rel=5e-2)
    assert slopes[1] == pytest.approx(-2 * g @ y, rel=1e-2)


def test_sampler_matches_exact_distribution():
    """Visit frequencies of the Metropolis chains against exact |Psi|^2 on
    the 2x2 lattice (36 configurations), blocking over walkers."""
    wl = inputs.hubbard("chi", 2, 2, 2, 2, "pair", seed=61, n_walkers=256)
    P = oracle.Problem(wl)
    occ_all, w = P.enumerate()
    key = {tuple(o): i for i, o in enumerate(occ_all)}
    occ = wl.init_occ.copy()
    step = np.zeros(wl.n_walkers, np.uint64)
    spw = 64
    samples, _, acc = P.sample(occ, step, 1234, 20, spw)
    assert acc.sum() > 0
    ids = np.array([key[tuple(o)] for o in samples]).reshape(wl.n_walkers, spw)
    hist = np.zeros((wl.n_walkers, len(w)))
    for k in range(wl.n_walkers):
        hist[k] = np.bincount(ids[k], minlength=len(w)) / spw
    p_hat = hist.mean(0)
    var = hist.var(0, ddof=1) / wl.n_walkers
    m = var > 0
    chi2 = np.sum((p_hat[m] - w[m]) ** 2 / var[m])
    dof = m.sum()
    assert chi2 < dof + 6 * np.sqrt(2 * dof)
    assert np.abs(p_hat - w).sum() < 0.05


def test_sampler_is_deterministic_and_resumable():
    wl = inputs.hubbard("det", 3, 2, 2, 2, "pair", seed=71, n_walkers=8)
    P = oracle.Problem(wl)
    o1, s1 = wl.init_occ.copy(), np.zeros(8, np.uint64)
    a, _, _ = P.sample(o1, s1, 5, 4, 6)
    o2, s2 = wl.init_occ.copy(), np.zeros(8, np.uint64)
    b1, _, _ = P.sample(o2, s2, 5, 4, 3)
    b2, _, _ = P.sample(o2, s2, 5, 0, 3)
    # resuming the chains reproduces the same samples
    a = a.reshape(8, 6, -1)
    b = np.concatenate([b1.reshape(8, 3, -1), b2.reshape(8, 3, -1)], axis=1)
    assert np.array_equal(a, b)
    assert np.array_equal(o1, o2) and np.array_equal(s1, s2)
    assert (s1 == (4 + 6) * wl.N).all()
