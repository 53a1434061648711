"""Pins of the oracle's accelerated linear method (Sec. II.B, Eq. 8-10).

The paper gives no numbers for the linear method (it was not run), so every
pin is a fact of the mathematics: the factored Hamiltonian of Eq. 9 must be
the Jordan-Wigner Hamiltonian itself; with exact |Psi|^2 weights the Eq. 10
product must be <Psi^i|H|Psi^j> x_j built from explicit vectors; on a
complete basis the lowest eigenvalue must be the exact ground energy; the
Davidson iteration must agree with a dense generalized eigensolver.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp

import oracle
from paper_1108_0900_gb300 import inputs


def _jw(M):
    """a_p as 2^M x 2^M sparse matrices (bit p = occupation of orbital p,
    sign = parity of the occupied orbitals below p)."""
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


def _jw_hamiltonian(wl, a, ad):
    """H of the workload from its definition (bond list / integrals)."""
    n = wl.n_sites
    H = 0 * a[0]
    if wl.ham == inputs.HUBBARD:
        for (i, j), t in zip(wl.bonds, wl.bond_t):
            if i == j:
                continue
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
        for s1, s2 in itertools.product(range(2), repeat=2):
            for p, q, r, s in itertools.product(range(n), repeat=4):
                if eri[p, q, r, s] != 0.0:
                    H = H + 0.5 * eri[p, q, r, s] * (ad[s1 * n + p] @ ad[s2 * n + r] @ a[s2 * n + s]
                                                     @ a[s1 * n + q])
    return H


def _bits(occ):
    return sum(1 << int(o) for o in occ)


CASES = {
    "hubbard2x2": lambda: inputs.hubbard("t", 2, 2, 2, 2, "2x2", seed=3, n_walkers=4, samples_per_walker=3),
    "hubbard3x2_pair": lambda: inputs.hubbard("t", 3, 2, 2, 2, "pair", seed=5, n_walkers=4, samples_per_walker=3),
    "abinitio4": lambda: inputs.abinitio("t", 4, 2, 2, n_chol=5, seed=6, n_walkers=4, samples_per_walker=3),
    "abinitio3": lambda: inputs.abinitio("t", 3, 1, 1, n_chol=4, seed=4, n_walkers=4, samples_per_walker=3),
}


@pytest.mark.parametrize("kind", list(CASES))
def test_factored_hamiltonian_is_the_hamiltonian(kind):
    """Eq. 9 with the readings of lm_factors: c0 + sum_mu Lhat_mu Rhat_mu
    equals the Jordan-Wigner Hamiltonian on the (N_up, N_dn) sector."""
    wl = CASES[kind]()
    M, n = wl.M, wl.n_sites
    a = _jw(M)
    ad = [x.T.tocsr() for x in a]
    Lf, Rf, c0 = oracle.lm_factors(wl)
    E = [[sum(ad[s * n + i] @ a[s * n + j] for s in range(2)) for j in range(n)] for i in range(n)]

    def one_body(K):
        out = 0 * a[0]
        for i in range(n):
            for j in range(n):
                if K[i, j] != 0.0:
                    out = out + K[i, j] * E[i][j]
        return out

    Hf = c0 * sp.identity(1 << M, format="csr")
    for Lm, Rm in zip(Lf, Rf):
        Hf = Hf + one_body(Lm) @ one_body(Rm)
    H = _jw_hamiltonian(wl, a, ad)
    P = oracle.Problem(wl)
    occ_all, _ = P.enumerate()
    idx = [_bits(o) for o in occ_all]
    A = H.toarray()[np.ix_(idx, idx)]
    B = Hf.toarray()[np.ix_(idx, idx)]
    assert np.abs(A - B).max() < 1e-12 * max(1.0, np.abs(A).max())


def _dense_lm(P, wl):
    """<Psi^i|H|Psi^j> / <Psi|Psi> and <Psi^i|Psi^j> / <Psi|Psi> over the
    sector from explicit vectors Psi^0 = Psi, Psi^j_n = Psi_n O_j(n) and
    the Jordan-Wigner H."""
    M = wl.M
    a = _jw(M)
    ad = [x.T.tocsr() for x in a]
    occ_all, w = P.enumerate()
    idx = [_bits(o) for o in occ_all]
    H = _jw_hamiltonian(wl, a, ad).toarray()[np.ix_(idx, idx)]
    psi = np.array([np.exp(l) * s for l, s in (P.log_psi(o) for o in occ_all)])
    O = np.array([P.logderiv(o) for o in occ_all])
    Psi = np.column_stack([psi, psi[:, None] * O])          # [n_conf, n_v + 1]
    nrm = psi @ psi
    return occ_all, w, Psi.T @ H @ Psi / nrm, Psi.T @ Psi / nrm


@pytest.mark.parametrize("kind", list(CASES))
def test_eq10_product_with_exact_weights_is_the_dense_matrix(kind):
    """Sampling n from |Psi_n|^2 exactly (enumeration weights), the Eq. 10
    right-to-left product reproduces H_ij x_j and S_ij x_j of the explicit
    basis vectors, for random x."""
    wl = CASES[kind]()
    P = oracle.Problem(wl)
    occ_all, w, Hd, Sd = _dense_lm(P, wl)
    fac = oracle.lm_factors(wl)
    rng = np.random.default_rng(1)
    for _ in range(2):
        x = rng.standard_normal(P.n_params() + 1)
        Hx, Sx = P.lm_apply(occ_all, fac, x, weights=w)
        assert np.linalg.norm(Hx - Hd @ x) <= 1e-10 * np.linalg.norm(Hd @ x)
        assert np.linalg.norm(Sx - Sd @ x) <= 1e-10 * np.linalg.norm(Sd @ x)
    # column 0 row 0: the variational energy sum_n w_n E_L(n)
    E, _ = P.measure(occ_all, want_O=False)
    e0 = np.zeros(P.n_params() + 1)
    e0[0] = 1.0
    Hx, Sx = P.lm_apply(occ_all, fac, e0, weights=w)
    assert Hx[0] == pytest.approx(np.sum(w * E), rel=1e-10)
    assert Sx[0] == pytest.approx(1.0, rel=1e-12)


def _columns(P, occ, fac, nv1, weights=None):
    H = np.zeros((nv1, nv1))
    S = np.zeros((nv1, nv1))
    for j in range(nv1):
        e = np.zeros(nv1)
        e[j] = 1.0
        H[:, j], S[:, j] = P.lm_apply(occ, fac, e, weights=weights)
    return H, S


def test_sampled_matrices_are_symmetric_and_S_is_the_plain_moment():
    """With sampled configurations the factored form (one-body terms split
    as (K Nhat + Nhat K) / 2N) gives a symmetric H estimate; S is
    (1/n) sum_n (1, O(n)) (1, O(n))^T from the measured O rows."""
    wl = inputs.abinitio("t", 3, 1, 1, n_chol=3, seed=8, n_walkers=6, samples_per_walker=2)
    P = oracle.Problem(wl)
    occ = wl.init_occ
    fac = oracle.lm_factors(wl)
    nv1 = P.n_params() + 1
    H, S = _columns(P, occ, fac, nv1)
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()
    _, O = P.measure(occ)
    o = np.column_stack([np.ones(len(occ)), O])
    assert np.abs(S - o.T @ o / len(occ)).max() <= 1e-13


def test_davidson_matches_dense_generalized_eigensolver():
    """The Davidson iteration on the Eq. 10 products (their dense columns,
    512 samples, 259 parameters) reaches the lowest eigenpair of a dense
    generalized symmetric eigensolver."""
    nw = 256
    wl = inputs.hubbard("t", 3, 2, 2, 2, "pair", seed=9, n_walkers=nw, samples_per_walker=2)
    P = oracle.Problem(wl)
    occ, _, _ = P.sample(wl.init_occ.copy(), np.zeros(nw, np.uint64), 5, 20, 2)
    fac = oracle.lm_factors(wl)
    nv1 = P.n_params() + 1
    H, S = _columns(P, occ, fac, nv1)
    a_shift, eps = 1.0, 1e-2
    D = np.eye(nv1)
    D[0, 0] = 0.0
    lam, vec = scipy.linalg.eigh(0.5 * (H + H.T) + a_shift * D, 0.5 * (S + S.T) + eps * D)
    theta, x, it, rel = oracle.lm_davidson(lambda v: (H @ v, S @ v), np.diag(S).copy(),
                                           a_shift, eps, tol=1e-10, max_iter=1000, max_sub=40)
    assert rel <= 1e-10
    assert theta == pytest.approx(lam[0], rel=1e-9)
    ref = vec[:, 0] / vec[0, 0]
    assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref)


def test_complete_basis_gives_the_exact_ground_energy():
    """Two sites, one up + one down electron, one correlator on both sites:
    every configuration has its own correlator amplitude, so {Psi^j} spans
    the whole sector and the lowest eigenvalue of Eq. 8 (exact weights) is
    the exact ground energy (U - sqrt(U^2 + 16 t^2)) / 2."""
    U, t = 4.0, 1.0
    E0 = (U - np.sqrt(U * U + 16 * t * t)) / 2
    rng = np.random.default_rng(3)
    wl = inputs.Workload(name="2site", n_sites=2, n_up=1, n_dn=1, ham=inputs.HUBBARD,
                         corr_sites=[np.array([0, 1], np.int32)], C=1.0 + 0.3 * rng.standard_normal(16),
                         f=np.array([0.3, 0.7, -0.4, 0.9, 0.5, 0.2]),
                         bonds=np.array([[0, 1]], np.int32), bond_t=np.array([t]), U=U)
    P = oracle.Problem(wl)
    occ_all, w = P.enumerate()
    fac = oracle.lm_factors(wl)
    nv1 = P.n_params() + 1
    H, S = _columns(P, occ_all, fac, nv1, weights=w)
    # restrict to the range of S (the basis is redundant) and solve there
    ev, U_ = np.linalg.eigh(0.5 * (S + S.T))
    keep = ev > 1e-10 * ev.max()
    B = U_[:, keep] / np.sqrt(ev[keep])
    lam = np.linalg.eigvalsh(B.T @ (0.5 * (H + H.T)) @ B)
    assert keep.sum() == 4
    assert lam[0] == pytest.approx(E0, abs=1e-10)
    # the energy before the step is above it
    E, _ = P.measure(occ_all, want_O=False)
    assert np.sum(w * E) > E0 + 1e-3


def test_update_moves_downhill():
    """alpha' = alpha + x_{1:} / (S x)_0: for small steps along the update the
    exact energy decreases (its slope 2 g . dalpha is negative)."""
    wl = inputs.hubbard("t", 2, 2, 2, 2, "pair", seed=12, n_walkers=4, samples_per_walker=3)
    P = oracle.Problem(wl)
    occ_all, w = P.enumerate()
    fac = oracle.lm_factors(wl)
    nv1 = P.n_params() + 1
    H, S = _columns(P, occ_all, fac, nv1, weights=w)
    eps, a_shift = 1e-3, 0.5
    theta, x, it, rel = oracle.lm_davidson(lambda v: P.lm_apply(occ_all, fac, v, weights=w),
                                           np.diag(S).copy(), a_shift, eps, tol=1e-10, max_iter=400)
    _, Sx = P.lm_apply(occ_all, fac, x, weights=w)
    alpha = np.concatenate([wl.C, wl.f])
    dalpha = oracle.lm_update(alpha, x, Sx[0]) - alpha
    E, O = P.measure(occ_all)
    g = O.T @ (w * E) - np.sum(w * E) * (O.T @ w)
    assert g @ dalpha < 0.0
    assert theta < np.sum(w * E)
