/*
 * Plain FP64 CPU oracle for the matrix-free stochastic-reconfiguration (SR)
 * hot path of a correlator-product-state x pfaffian wavefunction
 * (Neuscamman, Umrigar, Chan, "Optimizing large parameter sets in variational
 * quantum Monte Carlo", arXiv:1108.0900).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference the CUDA library is checked against.  Only the test suite, the
 * package smoke check and the CPU-baseline leg of the benchmark may load it;
 * the product path never calls it and shares no code with it.
 *
 * Everything is written for clarity, not speed: amplitudes are recomputed
 * from scratch (a fresh pfaffian for every configuration), derivative-ratio
 * vectors are dense of length n_v, and S is applied exactly as written in
 * Eq. 7.  Where the paper is silent the readings are:
 *   - spin orbital p = sigma * n_sites + site; occupied lists are ascending;
 *   - correlator local state idx_c = sum_j 4^j (n_{s_j,up} + 2 n_{s_j,dn});
 *   - Hubbard H = -sum_bonds t (c+_i c_j + c+_j c_i) (both spins)
 *                 + U sum_i n_iup n_idn, bond list taken as given;
 *   - Metropolis proposal: the a-th occupied orbital (ascending) moves to the
 *     k-th empty orbital of the same spin (ascending), a and k uniform from
 *     Philox4x32-10; accept iff u < |Psi'/Psi|^2;
 *   - S is the covariance form obtained by eliminating x_0 from Eq. 2 with
 *     O_0 = 1; all sample means use weight 1/n_s; shift eps is absolute.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random        */
/* numbers: as easy as 1, 2, 3").  Written from the published definition.   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra on small matrices                                   */
/* ------------------------------------------------------------------------ */

/* Pfaffian of an antisymmetric n x n matrix (row-major, destroyed), by the
 * Parlett-Reid reduction with pivoting described by Wimmer (the pfaffian
 * reference of Sec. II.C).  Returns sign in *sign and log|Pf| in *logabs;
 * a singular matrix gives sign 0. */
void orc_pfaffian(int n, double* A, double* logabs, int* sign)
{
    *logabs = 0.0;
    *sign = 1;
    if (n % 2) { *sign = 0; return; }
    for (int k = 0; k < n - 1; k += 2) {
        /* bring the largest entry of column k (below the diagonal) to k+1 */
        int kp = k + 1;
        double best = fabs(A[(k + 1) * n + k]);
        for (int i = k + 2; i < n; ++i) {
            if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); kp = i; }
        }
        if (kp != k + 1) {
            for (int j = 0; j < n; ++j) {
                double t = A[(k + 1) * n + j]; A[(k + 1) * n + j] = A[kp * n + j]; A[kp * n + j] = t;
            }
            for (int i = 0; i < n; ++i) {
                double t = A[i * n + k + 1]; A[i * n + k + 1] = A[i * n + kp]; A[i * n + kp] = t;
            }
            *sign = -*sign;
        }
        double piv = A[k * n + k + 1];
        if (piv == 0.0) { *sign = 0; *logabs = -INFINITY; return; }
        if (piv < 0) *sign = -*sign;
        *logabs += log(fabs(piv));
        /* congruence that clears row/column k beyond k+1:
           A[i][j] += tau_i A[j][k+1] - A[i][k+1] tau_j, tau_i = A[k][i] / A[k][k+1] */
        for (int i = k + 2; i < n; ++i) {
            double tau_i = A[k * n + i] / piv;
            for (int j = k + 2; j < n; ++j) {
                double tau_j = A[k * n + j] / piv;
                A[i * n + j] += tau_i * A[j * n + k + 1] - A[i * n + k + 1] * tau_j;
            }
        }
        /* the trailing block stays antisymmetric; k+2.. rows of column k+1 are
           not needed below because row k now has a single nonzero at k+1 */
    }
}

/* Inverse of a general n x n matrix (row-major) by Gauss-Jordan elimination
 * with partial pivoting.  Returns 0 on success, -1 if singular. */
int orc_inverse(int n, const double* A_in, double* X)
{
    double* A = (double*)malloc(sizeof(double) * n * n);
    memcpy(A, A_in, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) X[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int c = 0; c < n; ++c) {
        int pr = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[pr * n + c])) pr = r;
        if (A[pr * n + c] == 0.0) { free(A); return -1; }
        if (pr != c) {
            for (int j = 0; j < n; ++j) {
                double t = A[c * n + j]; A[c * n + j] = A[pr * n + j]; A[pr * n + j] = t;
                t = X[c * n + j]; X[c * n + j] = X[pr * n + j]; X[pr * n + j] = t;
            }
        }
        double d = A[c * n + c];
        for (int j = 0; j < n; ++j) { A[c * n + j] /= d; X[c * n + j] /= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double m = A[r * n + c];
            if (m == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                A[r * n + j] -= m * A[c * n + j];
                X[r * n + j] -= m * X[c * n + j];
            }
        }
    }
    free(A);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Parameter layout and wavefunction (Eq. 11)                               */
/* ------------------------------------------------------------------------ */

static int n_orb_M(const orc_problem* P) { return 2 * P->n_sites; }

static void corr_offsets(const orc_problem* P, int64_t* off);

int64_t orc_n_corr_params(const orc_problem* P)
{
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (P->n_corr + 1));
    corr_offsets(P, off);
    int64_t n = off[P->n_corr];
    free(off);
    return n;
}

int64_t orc_n_params(const orc_problem* P)
{
    int M = n_orb_M(P);
    return orc_n_corr_params(P) + (int64_t)M * (M - 1) / 2;
}

/* index of f_pq (p < q) in the row-major upper triangle */
static int64_t pf_index(int M, int p, int q)
{
    return (int64_t)p * M - (int64_t)p * (p + 1) / 2 + (q - p - 1);
}

static void occ_to_bits(const orc_problem* P, const uint8_t* occ, uint8_t* bits)
{
    int M = n_orb_M(P), N = P->n_up + P->n_dn;
    memset(bits, 0, M);
    for (int a = 0; a < N; ++a) bits[occ[a]] = 1;
}

/* local state of correlator c: sum_j 4^j (n_{s_j up} + 2 n_{s_j dn}) */
static int64_t corr_state(const orc_problem* P, const uint8_t* bits, int c)
{
    int64_t idx = 0, w = 1;
    for (int j = P->corr_ptr[c]; j < P->corr_ptr[c + 1]; ++j) {
        int s = P->corr_sites[j];
        idx += w * (bits[s] + 2 * bits[P->n_sites + s]);
        w *= 4;
    }
    return idx;
}

int64_t orc_corr_state(const orc_problem* P, const uint8_t* occ, int c)
{
    uint8_t bits[512];
    occ_to_bits(P, occ, bits);
    return corr_state(P, bits, c);
}

/* off[c] = parameter index of state 0 of correlator c; off[n_corr] = number
 * of correlator parameters.  Each class owns one block of 4^m parameters,
 * classes in index order; a correlator reads its class's block. */
static void corr_offsets(const orc_problem* P, int64_t* off)
{
    if (!P->corr_class) {
        off[0] = 0;
        for (int c = 0; c < P->n_corr; ++c) {
            int m = P->corr_ptr[c + 1] - P->corr_ptr[c];
            off[c + 1] = off[c] + ((int64_t)1 << (2 * m));
        }
        return;
    }
    int n_class = 0;
    for (int c = 0; c < P->n_corr; ++c)
        if (P->corr_class[c] + 1 > n_class) n_class = P->corr_class[c] + 1;
    int64_t* cls = (int64_t*)calloc((size_t)n_class + 1, sizeof(int64_t));
    for (int c = 0; c < P->n_corr; ++c) {
        int m = P->corr_ptr[c + 1] - P->corr_ptr[c];
        cls[P->corr_class[c] + 1] = (int64_t)1 << (2 * m);
    }
    for (int q = 0; q < n_class; ++q) cls[q + 1] += cls[q];
    for (int c = 0; c < P->n_corr; ++c) off[c] = cls[P->corr_class[c]];
    off[P->n_corr] = cls[n_class];
    free(cls);
}

/* A = F[occ, occ] with F_pq = f_pq (p < q), F_qp = -f_pq, F_pp = 0 */
static void pairing_submatrix(const orc_problem* P, const uint8_t* occ, double* A)
{
    int M = n_orb_M(P), N = P->n_up + P->n_dn;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            int p = occ[a], q = occ[b];
            double v = 0.0;
            if (p < q) v = P->f[pf_index(M, p, q)];
            else if (p > q) v = -P->f[pf_index(M, q, p)];
            A[a * N + b] = v;
        }
}

/* log|Psi_n| and sign of Psi_n = prod_c C_c[idx_c(n)] * Pf(F[occ, occ])
 * (Eq. 11, with the correlators acting diagonally on the pfaffian). */
void orc_log_psi(const orc_problem* P, const uint8_t* occ, double* logabs, int* sign)
{
    int N = P->n_up + P->n_dn;
    uint8_t bits[512];
    occ_to_bits(P, occ, bits);
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (P->n_corr + 1));
    corr_offsets(P, off);
    double la = 0.0;
    int sg = 1;
    for (int c = 0; c < P->n_corr; ++c) {
        double v = P->C[off[c] + corr_state(P, bits, c)];
        if (v == 0.0) { sg = 0; la = -INFINITY; break; }
        if (v < 0) sg = -sg;
        la += log(fabs(v));
    }
    free(off);
    double* A = (double*)malloc(sizeof(double) * N * N);
    pairing_submatrix(P, occ, A);
    double lp;
    int sp;
    orc_pfaffian(N, A, &lp, &sp);
    free(A);
    *logabs = la + lp;
    *sign = sg * sp;
}

/* Dense derivative-ratio vector O_k(n) = (dPsi_n/dalpha_k)/Psi_n (Eq. 3):
 * correlator part 1/C_c[idx_c] at its own parameter; pairing part
 * (A^{-1})_{b a} for f_pq with p = occ[a] < q = occ[b] (d ln Pf(A)/dA_ab).
 * O has length n_v.  Returns -1 if A is singular. */
int orc_logderiv(const orc_problem* P, const uint8_t* occ, double* O)
{
    int M = n_orb_M(P), N = P->n_up + P->n_dn;
    int64_t ncp = orc_n_corr_params(P), nv = orc_n_params(P);
    memset(O, 0, sizeof(double) * nv);
    uint8_t bits[512];
    occ_to_bits(P, occ, bits);
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (P->n_corr + 1));
    corr_offsets(P, off);
    for (int c = 0; c < P->n_corr; ++c) {
        int64_t k = off[c] + corr_state(P, bits, c);
        O[k] += 1.0 / P->C[k];
    }
    free(off);
    double* A = (double*)malloc(sizeof(double) * N * N);
    double* X = (double*)malloc(sizeof(double) * N * N);
    pairing_submatrix(P, occ, A);
    int rc = orc_inverse(N, A, X);
    if (rc == 0) {
        for (int a = 0; a < N; ++a)
            for (int b = a + 1; b < N; ++b)
                O[ncp + pf_index(M, occ[a], occ[b])] = X[b * N + a];
    }
    free(A);
    free(X);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Second quantisation helpers (explicit Jordan-Wigner signs)               */
/* ------------------------------------------------------------------------ */

/* apply a_q then a+_p to the ascending-ordered determinant `bits`; returns
 * the sign (0 if the result vanishes) and writes the new occupation. */
static int hop_sign(int M, const uint8_t* bits, int p, int q, uint8_t* out)
{
    if (!bits[q]) return 0;
    memcpy(out, bits, M);
    int s = 1;
    for (int o = 0; o < q; ++o) if (out[o]) s = -s;
    out[q] = 0;
    if (out[p]) return 0;
    for (int o = 0; o < p; ++o) if (out[o]) s = -s;
    out[p] = 1;
    return s;
}

static void bits_to_occ(int M, const uint8_t* bits, uint8_t* occ)
{
    int a = 0;
    for (int o = 0; o < M; ++o) if (bits[o]) occ[a++] = (uint8_t)o;
}

/* Psi_{n'} / Psi_n from two fresh amplitude evaluations */
static double amp_ratio(const orc_problem* P, const uint8_t* occ_new, double la0, int s0)
{
    double la;
    int s;
    orc_log_psi(P, occ_new, &la, &s);
    if (s == 0) return 0.0;
    return (double)(s * s0) * exp(la - la0);
}

/* Local energy E_L(n) = sum_n' <n|H|n'> Psi_n'/Psi_n (the quantity implied by
 * <Psi^i|H|Psi> in Eq. 2), Hubbard model, every Psi_n' recomputed from
 * scratch and every matrix element signed explicitly. */
double orc_local_energy_hubbard(const orc_problem* P, const uint8_t* occ)
{
    int M = n_orb_M(P), N = P->n_up + P->n_dn, ns = P->n_sites;
    uint8_t bits[512], nb[512], occn[256];
    occ_to_bits(P, occ, bits);
    double la0;
    int s0;
    orc_log_psi(P, occ, &la0, &s0);
    double E = 0.0;
    for (int i = 0; i < ns; ++i) E += P->U * bits[i] * bits[ns + i];
    for (int b = 0; b < P->n_bonds; ++b) {
        int i = P->bonds[2 * b], j = P->bonds[2 * b + 1];
        double t = P->bond_t[b];
        if (i == j) continue;
        for (int sg = 0; sg < 2; ++sg) {
            for (int dir = 0; dir < 2; ++dir) {
                /* term -t a+_x a_y; <n| a+_x a_y |n'> is nonzero for
                   n' = n with the electron moved x -> y */
                int x = sg * ns + (dir ? j : i);
                int y = sg * ns + (dir ? i : j);
                if (!bits[x] || bits[y]) continue;
                memcpy(nb, bits, M);
                nb[x] = 0;
                nb[y] = 1;
                uint8_t back[512];
                int me = hop_sign(M, nb, x, y, back); /* <n|a+_x a_y|n'> */
                if (me == 0) continue;
                bits_to_occ(M, nb, occn);
                E += -t * me * amp_ratio(P, occn, la0, s0);
            }
        }
    }
    (void)N;
    return E;
}

/* One- and two-electron matrix element <n|H|n'> for the ab initio
 * Hamiltonian H = sum_{pq,s} h_pq a+_ps a_qs
 *               + 1/2 sum_{pqrs,st} (pq|rs) a+_ps a+_rt a_st a_qs,
 * (pq|rs) = sum_mu L^mu_pq L^mu_rs  (Eq. 9 with R = L).
 * Evaluated by applying every operator string to |n'> with explicit signs:
 * slow, only used on small tests. */
static double eri(const orc_problem* P, int p, int q, int r, int s)
{
    int n = P->n_sites;
    double v = 0.0;
    for (int mu = 0; mu < P->n_chol; ++mu)
        v += P->chol[(size_t)mu * n * n + p * n + q] * P->chol[(size_t)mu * n * n + r * n + s];
    return v;
}

static int apply_annihilate(int M, uint8_t* bits, int q)
{
    if (!bits[q]) return 0;
    int s = 1;
    for (int o = 0; o < q; ++o) if (bits[o]) s = -s;
    bits[q] = 0;
    return s;
}

static int apply_create(int M, uint8_t* bits, int p)
{
    if (bits[p]) return 0;
    int s = 1;
    for (int o = 0; o < p; ++o) if (bits[o]) s = -s;
    bits[p] = 1;
    return s;
}

double orc_hamiltonian_element(const orc_problem* P, const uint8_t* occ_n, const uint8_t* occ_np)
{
    int M = n_orb_M(P), n = P->n_sites;
    uint8_t bn[512], bnp[512], w[512];
    occ_to_bits(P, occ_n, bn);
    occ_to_bits(P, occ_np, bnp);
    double H = 0.0;
    if (P->ham == 0) {
        int same = memcmp(bn, bnp, M) == 0;
        if (same) for (int i = 0; i < n; ++i) H += P->U * bn[i] * bn[n + i];
        for (int b = 0; b < P->n_bonds; ++b) {
            int i = P->bonds[2 * b], j = P->bonds[2 * b + 1];
            if (i == j) continue;
            for (int sg = 0; sg < 2; ++sg)
                for (int dir = 0; dir < 2; ++dir) {
                    int x = sg * n + (dir ? j : i), y = sg * n + (dir ? i : j);
                    memcpy(w, bnp, M);
                    int s = apply_annihilate(M, w, y);
                    if (!s) continue;
                    int s2 = apply_create(M, w, x);
                    if (!s2) continue;
                    if (memcmp(w, bn, M) == 0) H += -P->bond_t[b] * s * s2;
                }
        }
        return H;
    }
    for (int s1 = 0; s1 < 2; ++s1)
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                memcpy(w, bnp, M);
                int s = apply_annihilate(M, w, s1 * n + q);
                if (!s) continue;
                int s2 = apply_create(M, w, s1 * n + p);
                if (!s2) continue;
                if (memcmp(w, bn, M) == 0) H += P->h[p * n + q] * s * s2;
            }
    for (int s1 = 0; s1 < 2; ++s1)
        for (int s2 = 0; s2 < 2; ++s2)
            for (int p = 0; p < n; ++p)
                for (int q = 0; q < n; ++q)
                    for (int r = 0; r < n; ++r)
                        for (int s = 0; s < n; ++s) {
                            /* a+_{p s1} a+_{r s2} a_{s s2} a_{q s1} acting on |n'> */
                            memcpy(w, bnp, M);
                            int g = apply_annihilate(M, w, s1 * n + q);
                            if (!g) continue;
                            int g2 = apply_annihilate(M, w, s2 * n + s);
                            if (!g2) continue;
                            int g3 = apply_create(M, w, s2 * n + r);
                            if (!g3) continue;
                            int g4 = apply_create(M, w, s1 * n + p);
                            if (!g4) continue;
                            if (memcmp(w, bn, M) == 0) H += 0.5 * eri(P, p, q, r, s) * g * g2 * g3 * g4;
                        }
    return H;
}

/* One two-body string 1/2 (pq|rs) a+_{p} a+_{r} a_{s} a_{q} (spin orbitals,
 * spins of p,q equal and of r,s equal, spatial integrals) applied to |n'>:
 * returns its coefficient on |n> (0 if it does not land on n). */
static double two_body_term(const orc_problem* P, const uint8_t* bn, const uint8_t* bnp, int p, int q, int r, int s)
{
    int M = n_orb_M(P), n = P->n_sites;
    if ((p >= n) != (q >= n) || (r >= n) != (s >= n)) return 0.0;
    uint8_t w[512];
    memcpy(w, bnp, M);
    int g = apply_annihilate(M, w, q);
    if (!g) return 0.0;
    int g2 = apply_annihilate(M, w, s);
    if (!g2) return 0.0;
    int g3 = apply_create(M, w, r);
    if (!g3) return 0.0;
    int g4 = apply_create(M, w, p);
    if (!g4) return 0.0;
    if (memcmp(w, bn, M) != 0) return 0.0;
    return 0.5 * eri(P, p % n, q % n, r % n, s % n) * g * g2 * g3 * g4;
}

static double one_body_term(const orc_problem* P, const uint8_t* bn, const uint8_t* bnp, int p, int q)
{
    int M = n_orb_M(P), n = P->n_sites;
    if ((p >= n) != (q >= n)) return 0.0;
    uint8_t w[512];
    memcpy(w, bnp, M);
    int g = apply_annihilate(M, w, q);
    if (!g) return 0.0;
    int g2 = apply_create(M, w, p);
    if (!g2) return 0.0;
    if (memcmp(w, bn, M) != 0) return 0.0;
    return P->h[(p % n) * n + (q % n)] * g * g2;
}

/* <n|H|n'> for the ab initio Hamiltonian, applying to |n'> only the operator
 * strings that can connect it to |n> (every other string of H maps |n'> to a
 * configuration other than |n>, or to zero).  `rem` = orbitals of n' not in
 * n (annihilated), `add` = orbitals of n not in n' (created), `nd` = how many
 * (0, 1 or 2); the remaining indices run over occupied spectators. */
static double abinitio_element(const orc_problem* P, const uint8_t* bn, const uint8_t* bnp, const int* rem,
                               const int* add, int nd)
{
    int M = n_orb_M(P);
    double H = 0.0;
    if (nd == 0) {
        for (int k = 0; k < M; ++k) {
            if (!bnp[k]) continue;
            H += one_body_term(P, bn, bnp, k, k);
            for (int l = 0; l < M; ++l) {
                if (!bnp[l] || l == k) continue;
                H += two_body_term(P, bn, bnp, k, k, l, l);   /* direct */
                H += two_body_term(P, bn, bnp, l, k, k, l);   /* exchange */
            }
        }
    } else if (nd == 1) {
        int i = rem[0], a = add[0];
        H += one_body_term(P, bn, bnp, a, i);
        for (int k = 0; k < M; ++k) {
            if (!bnp[k] || k == i) continue;
            H += two_body_term(P, bn, bnp, a, i, k, k);
            H += two_body_term(P, bn, bnp, k, k, a, i);
            H += two_body_term(P, bn, bnp, a, k, k, i);
            H += two_body_term(P, bn, bnp, k, i, a, k);
        }
    } else {
        int i = rem[0], j = rem[1], a = add[0], b = add[1];
        int qs[2][2] = {{i, j}, {j, i}}, pr[2][2] = {{a, b}, {b, a}};
        for (int u = 0; u < 2; ++u)
            for (int v = 0; v < 2; ++v)
                H += two_body_term(P, bn, bnp, pr[v][0], qs[u][0], pr[v][1], qs[u][1]);
    }
    return H;
}

/* Local energy for the ab initio Hamiltonian: every configuration n' reached
 * by moving one or two electrons (spin kept), <n|H|n'> by explicit operator
 * application (abinitio_element) and Psi_n' from scratch. */
double orc_local_energy_abinitio(const orc_problem* P, const uint8_t* occ)
{
    int M = n_orb_M(P), N = P->n_up + P->n_dn, n = P->n_sites;
    uint8_t bits[512], w[512], occn[256];
    occ_to_bits(P, occ, bits);
    double la0;
    int s0;
    orc_log_psi(P, occ, &la0, &s0);
    double E = abinitio_element(P, bits, bits, NULL, NULL, 0);
    int occl[256], empl[256];
    int nocc = 0, nemp = 0;
    for (int o = 0; o < M; ++o) { if (bits[o]) occl[nocc++] = o; else empl[nemp++] = o; }
    for (int a = 0; a < nocc; ++a)
        for (int e = 0; e < nemp; ++e) {
            if ((occl[a] >= n) != (empl[e] >= n)) continue;
            memcpy(w, bits, M);
            w[occl[a]] = 0; w[empl[e]] = 1;
            /* n' = n with occl[a] -> empl[e]; n' has empl[e] where n has occl[a] */
            int rem[1] = {empl[e]}, add[1] = {occl[a]};
            double h = abinitio_element(P, bits, w, rem, add, 1);
            if (h != 0.0) {
                bits_to_occ(M, w, occn);
                E += h * amp_ratio(P, occn, la0, s0);
            }
        }
    for (int a1 = 0; a1 < nocc; ++a1)
        for (int a2 = a1 + 1; a2 < nocc; ++a2)
            for (int e1 = 0; e1 < nemp; ++e1)
                for (int e2 = e1 + 1; e2 < nemp; ++e2) {
                    int up_out = (occl[a1] < n) + (occl[a2] < n);
                    int up_in = (empl[e1] < n) + (empl[e2] < n);
                    if (up_out != up_in) continue;
                    memcpy(w, bits, M);
                    w[occl[a1]] = 0; w[occl[a2]] = 0; w[empl[e1]] = 1; w[empl[e2]] = 1;
                    int rem[2] = {empl[e1], empl[e2]}, add[2] = {occl[a1], occl[a2]};
                    double h = abinitio_element(P, bits, w, rem, add, 2);
                    if (h != 0.0) {
                        bits_to_occ(M, w, occn);
                        E += h * amp_ratio(P, occn, la0, s0);
                    }
                }
    (void)N;
    return E;
}

/* The same local energy with every matrix element from the unrestricted
 * operator sum of orc_hamiltonian_element: slow, tiny systems only. */
double orc_local_energy_abinitio_bruteforce(const orc_problem* P, const uint8_t* occ)
{
    int M = n_orb_M(P), n = P->n_sites;
    uint8_t bits[512], w[512], occn[256];
    occ_to_bits(P, occ, bits);
    double la0;
    int s0;
    orc_log_psi(P, occ, &la0, &s0);
    double E = orc_hamiltonian_element(P, occ, occ);
    int occl[256], empl[256];
    int nocc = 0, nemp = 0;
    for (int o = 0; o < M; ++o) { if (bits[o]) occl[nocc++] = o; else empl[nemp++] = o; }
    for (int a = 0; a < nocc; ++a)
        for (int e = 0; e < nemp; ++e) {
            if ((occl[a] >= n) != (empl[e] >= n)) continue;
            memcpy(w, bits, M);
            w[occl[a]] = 0; w[empl[e]] = 1;
            bits_to_occ(M, w, occn);
            double h = orc_hamiltonian_element(P, occ, occn);
            if (h != 0.0) E += h * amp_ratio(P, occn, la0, s0);
        }
    for (int a1 = 0; a1 < nocc; ++a1)
        for (int a2 = a1 + 1; a2 < nocc; ++a2)
            for (int e1 = 0; e1 < nemp; ++e1)
                for (int e2 = e1 + 1; e2 < nemp; ++e2) {
                    int up_out = (occl[a1] < n) + (occl[a2] < n);
                    int up_in = (empl[e1] < n) + (empl[e2] < n);
                    if (up_out != up_in) continue;
                    memcpy(w, bits, M);
                    w[occl[a1]] = 0; w[occl[a2]] = 0; w[empl[e1]] = 1; w[empl[e2]] = 1;
                    bits_to_occ(M, w, occn);
                    double h = orc_hamiltonian_element(P, occ, occn);
                    if (h != 0.0) E += h * amp_ratio(P, occn, la0, s0);
                }
    return E;
}

double orc_local_energy(const orc_problem* P, const uint8_t* occ)
{
    return P->ham == 0 ? orc_local_energy_hubbard(P, occ) : orc_local_energy_abinitio(P, occ);
}

/* ------------------------------------------------------------------------ */
/* Metropolis sampling from |Psi_n|^2 / <Psi|Psi> in the fixed (N_up, N_dn)  */
/* sector (Sec. II.A, Eq. 3; sector restriction of Sec. III).               */
/* ------------------------------------------------------------------------ */

/* One proposal of walker w at step `step`.  Returns 1 if accepted and
 * updates occ in place; *margin receives |u - r^2| / r^2. */
static int metropolis_step(const orc_problem* P, uint8_t* occ, uint64_t seed, uint32_t walker,
                           uint64_t step, double* la, int* sg, double* margin)
{
    int M = n_orb_M(P), N = P->n_up + P->n_dn, ns = P->n_sites;
    uint32_t ctr[4] = {walker, (uint32_t)step, (uint32_t)(step >> 32), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    int a = (int)(((uint64_t)r[0] * (uint64_t)N) >> 32);
    int p = occ[a];
    int spin = p >= ns;
    int n_same = spin ? P->n_dn : P->n_up;
    int n_empty = ns - n_same;
    uint8_t bits[512], occn[256];
    occ_to_bits(P, occ, bits);
    if (n_empty <= 0) { *margin = INFINITY; return 0; }
    int k = (int)(((uint64_t)r[1] * (uint64_t)n_empty) >> 32);
    int q = -1;
    for (int o = spin * ns, seen = 0; o < (spin + 1) * ns; ++o) {
        if (!bits[o]) {
            if (seen == k) { q = o; break; }
            ++seen;
        }
    }
    double u = (double)(r[2] >> 8) * (1.0 / 16777216.0);
    bits[p] = 0;
    bits[q] = 1;
    bits_to_occ(M, bits, occn);
    double la1;
    int s1;
    orc_log_psi(P, occn, &la1, &s1);
    double ratio2 = (s1 == 0) ? 0.0 : exp(2.0 * (la1 - *la));
    *margin = ratio2 > 0 ? fabs(u - ratio2) / ratio2 : INFINITY;
    if (u < ratio2) {
        memcpy(occ, occn, N);
        *la = la1;
        *sg = s1;
        return 1;
    }
    return 0;
}

/* Run every walker's chain: n_burn sweeps, then n_spw sweeps each ending in
 * a stored sample; a sweep is N proposals.  occ [n_walkers][N] (ascending) and
 * step [n_walkers] are updated in place; samples go to
 * out_occ[(w * n_spw + j) * N + a]; min_margin[w] and accepts[w] are filled,
 * and first_close[w] is the index (within this call) of the first proposal
 * whose relative margin |u - r^2| / r^2 fell below close_tol, or -1. */
int orc_sample(const orc_problem* P, int n_walkers, uint8_t* occ, uint64_t* step,
               uint64_t seed, int n_burn, int n_spw, uint8_t* out_occ,
               double* min_margin, int64_t* accepts, double close_tol, int64_t* first_close)
{
    int N = P->n_up + P->n_dn;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
    for (int w = 0; w < n_walkers; ++w) {
        uint8_t* o = occ + (size_t)w * N;
        double la;
        int sg;
        orc_log_psi(P, o, &la, &sg);
        if (sg == 0) { bad++; continue; }
        double mm = INFINITY;
        int64_t acc = 0, fc = -1, k = 0;
        for (int sw = 0; sw < n_burn + n_spw; ++sw) {
            for (int t = 0; t < N; ++t, ++k) {
                double m;
                acc += metropolis_step(P, o, seed, (uint32_t)w, step[w], &la, &sg, &m);
                step[w]++;
                if (m < mm) mm = m;
                if (fc < 0 && m < close_tol) fc = k;
            }
            if (sw >= n_burn)
                memcpy(out_occ + ((size_t)w * n_spw + (sw - n_burn)) * N, o, N);
        }
        if (min_margin) min_margin[w] = mm;
        if (accepts) accepts[w] = acc;
        if (first_close) first_close[w] = fc;
    }
    return bad ? -1 : 0;
}

/* Local energy and dense derivative ratios for n_s given configurations. */
int orc_measure(const orc_problem* P, int64_t n_s, const uint8_t* occ, double* E, double* O)
{
    int N = P->n_up + P->n_dn;
    int64_t nv = orc_n_params(P);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : bad)
    for (int64_t s = 0; s < n_s; ++s) {
        if (E) E[s] = orc_local_energy(P, occ + s * N);
        if (O && orc_logderiv(P, occ + s * N, O + s * nv) != 0) bad++;
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* SR linear algebra on stored derivative ratios                            */
/* ------------------------------------------------------------------------ */

/* mean of O over samples (weight 1/n_s) */
void orc_mean_O(int64_t n_s, int64_t nv, const double* O, double* Obar)
{
    for (int64_t k = 0; k < nv; ++k) Obar[k] = 0.0;
    for (int64_t s = 0; s < n_s; ++s)
        for (int64_t k = 0; k < nv; ++k) Obar[k] += O[s * nv + k];
    for (int64_t k = 0; k < nv; ++k) Obar[k] /= (double)n_s;
}

/* g_k = <E_L O_k> - <E_L><O_k>: the right-hand side left after x_0 is
 * eliminated from Eq. 2 (up to the factor -tau). */
void orc_gradient(int64_t n_s, int64_t nv, const double* O, const double* E, double* g,
                  double* E_mean)
{
    double Em = 0.0;
    for (int64_t s = 0; s < n_s; ++s) Em += E[s];
    Em /= (double)n_s;
    double* Ob = (double*)malloc(sizeof(double) * nv);
    orc_mean_O(n_s, nv, O, Ob);
    for (int64_t k = 0; k < nv; ++k) g[k] = 0.0;
    for (int64_t s = 0; s < n_s; ++s)
        for (int64_t k = 0; k < nv; ++k) g[k] += E[s] * O[s * nv + k];
    for (int64_t k = 0; k < nv; ++k) g[k] = g[k] / (double)n_s - Em * Ob[k];
    free(Ob);
    if (E_mean) *E_mean = Em;
}

/* Dense S_ij = <O_i O_j> - <O_i><O_j> (Eq. 3 with the mean part removed);
 * S is nv x nv.  Only for small nv. */
void orc_dense_S(int64_t n_s, int64_t nv, const double* O, double* S)
{
    double* Ob = (double*)malloc(sizeof(double) * nv);
    orc_mean_O(n_s, nv, O, Ob);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nv; ++i) {
        for (int64_t j = 0; j < nv; ++j) {
            double acc = 0.0;
            for (int64_t s = 0; s < n_s; ++s) acc += O[s * nv + i] * O[s * nv + j];
            S[i * nv + j] = acc / (double)n_s - Ob[i] * Ob[j];
        }
    }
    free(Ob);
}

/* (S + eps I) v by the interchanged summation of Eq. 7:
 * out = (1/n_s) sum_s O_s (O_s . v) - Obar (Obar . v) + eps v. */
void orc_apply_S(int64_t n_s, int64_t nv, const double* O, const double* Obar, const double* v,
                 double eps, double* out)
{
    double ob_v = 0.0;
    for (int64_t k = 0; k < nv; ++k) ob_v += Obar[k] * v[k];
    for (int64_t k = 0; k < nv; ++k) out[k] = 0.0;
    for (int64_t s = 0; s < n_s; ++s) {
        const double* Os = O + s * nv;
        double t = 0.0;
        for (int64_t k = 0; k < nv; ++k) t += Os[k] * v[k];
        for (int64_t k = 0; k < nv; ++k) out[k] += Os[k] * t;
    }
    for (int64_t k = 0; k < nv; ++k) out[k] = out[k] / (double)n_s - Obar[k] * ob_v + eps * v[k];
}

/* Eq. 7 evaluated from compact per-sample rows, with v given for k vectors.
 * Sample s holds its ascending occupation occ[s][N], its correlator states
 * cs[s][n_corr] and the values of its n_pair pairing derivatives
 * pf[s][n_pair]; value e is O of f_pq with p = occ[a_e], q = occ[b_e],
 * (a_e, b_e) = (pairs[2e], pairs[2e+1]), a_e < b_e.  A correlator factor
 * C_c[n_c] contributes O = 1/C at parameter off_c + state (Eq. 3 for one
 * factor; correlators of one class add up on their shared amplitude); every
 * other entry of O_s is zero.  Obar_out[nv] receives the mean of these rows
 * (weight 1/n_s) and, for each of the k columns v_j = v[j nv ..],
 *   out_j = (1/n_s) sum_s O_s (O_s . v_j) - Obar (Obar . v_j) + eps v_j,
 * all in FP64, summed over the samples in order. */
void orc_apply_S_compact(const orc_problem* P, int64_t n_s, const uint8_t* occ, const int64_t* cs, int n_pair,
                         const int32_t* pairs, const double* pf, int k, const double* v, double eps,
                         double* out, double* Obar_out)
{
    const int M = n_orb_M(P), N = P->n_up + P->n_dn;
    const int64_t nv = orc_n_params(P), ncp = orc_n_corr_params(P);
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)P->n_corr + 1));
    corr_offsets(P, off);
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * ((size_t)P->n_corr + (size_t)n_pair + 1));
    double* val = (double*)malloc(sizeof(double) * ((size_t)P->n_corr + (size_t)n_pair + 1));
    double* t = (double*)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    for (int64_t i = 0; i < nv; ++i) Obar_out[i] = 0.0;
    for (int64_t i = 0; i < nv * k; ++i) out[i] = 0.0;
    for (int64_t s = 0; s < n_s; ++s) {
        /* the nonzero entries of O_s: (index, value) pairs */
        const uint8_t* o = occ + s * N;
        int n = 0;
        for (int c = 0; c < P->n_corr; ++c) {
            idx[n] = off[c] + cs[s * P->n_corr + c];
            val[n] = 1.0 / P->C[idx[n]];
            ++n;
        }
        for (int e = 0; e < n_pair; ++e) {
            idx[n] = ncp + pf_index(M, o[pairs[2 * e]], o[pairs[2 * e + 1]]);
            val[n] = pf[s * n_pair + e];
            ++n;
        }
        for (int i = 0; i < n; ++i) Obar_out[idx[i]] += val[i];
        for (int j = 0; j < k; ++j) {
            t[j] = 0.0;
            for (int i = 0; i < n; ++i) t[j] += val[i] * v[j * nv + idx[i]];
        }
        for (int j = 0; j < k; ++j)
            for (int i = 0; i < n; ++i) out[j * nv + idx[i]] += val[i] * t[j];
    }
    for (int64_t i = 0; i < nv; ++i) Obar_out[i] /= (double)n_s;
    for (int j = 0; j < k; ++j) {
        double ob_v = 0.0;
        for (int64_t i = 0; i < nv; ++i) ob_v += Obar_out[i] * v[j * nv + i];
        for (int64_t i = 0; i < nv; ++i)
            out[j * nv + i] = out[j * nv + i] / (double)n_s - Obar_out[i] * ob_v + eps * v[j * nv + i];
    }
    free(off); free(idx); free(val); free(t);
}

static double dot(int64_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Conjugate gradient on (S + eps I) x = g with x_0 = 0 (Sec. II.A: S is only
 * touched through products).  Stops when the recurrence residual satisfies
 * |r|/|g| <= tol or after max_iter products.  Reports the iterations and the
 * true relative residual |g - (S + eps I) x| / |g|. */
int orc_cg(int64_t n_s, int64_t nv, const double* O, const double* g, double eps, double tol,
           int max_iter, double* x, int* iters, double* true_rel_res)
{
    double* Ob = (double*)malloc(sizeof(double) * nv);
    double* r = (double*)malloc(sizeof(double) * nv);
    double* p = (double*)malloc(sizeof(double) * nv);
    double* Ap = (double*)malloc(sizeof(double) * nv);
    orc_mean_O(n_s, nv, O, Ob);
    for (int64_t k = 0; k < nv; ++k) { x[k] = 0.0; r[k] = g[k]; p[k] = g[k]; }
    double gn = sqrt(dot(nv, g, g));
    double rr = dot(nv, r, r);
    int it = 0;
    int conv = gn == 0.0;
    while (!conv && it < max_iter) {
        orc_apply_S(n_s, nv, O, Ob, p, eps, Ap);
        double alpha = rr / dot(nv, p, Ap);
        for (int64_t k = 0; k < nv; ++k) { x[k] += alpha * p[k]; r[k] -= alpha * Ap[k]; }
        double rr_new = dot(nv, r, r);
        ++it;
        if (sqrt(rr_new) <= tol * gn) { conv = 1; rr = rr_new; break; }
        double beta = rr_new / rr;
        rr = rr_new;
        for (int64_t k = 0; k < nv; ++k) p[k] = r[k] + beta * p[k];
    }
    orc_apply_S(n_s, nv, O, Ob, x, eps, Ap);
    double res = 0.0;
    for (int64_t k = 0; k < nv; ++k) { double d = g[k] - Ap[k]; res += d * d; }
    if (true_rel_res) *true_rel_res = gn > 0 ? sqrt(res) / gn : 0.0;
    if (iters) *iters = it;
    free(Ob); free(r); free(p); free(Ap);
    return conv ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* SR parameter update (Sec. II.A).  Eq. 2 projects (1 - tau H)|Psi> onto the */
/* span of |Psi> and its derivatives with coefficients x_0, x.  Its row 0,    */
/* divided by <Psi|Psi>, reads 1 - tau <E> = x_0 + sum_j Obar_j x_j; the     */
/* remaining rows reduce to S x = -tau g, so x = -tau y for the solution y of */
/* (S + eps) y = g.  The new parameters are alpha_k + x_k / x_0.              */
/* ------------------------------------------------------------------------ */

double orc_sr_update(int64_t nv, const double* alpha, const double* y, double tau, double E_mean,
                     const double* Obar, double* alpha_out)
{
    double ox = 0.0;
    for (int64_t k = 0; k < nv; ++k) ox += Obar[k] * (-tau * y[k]);
    const double x0 = 1.0 - tau * E_mean - ox;
    for (int64_t k = 0; k < nv; ++k) alpha_out[k] = alpha[k] + (-tau * y[k]) / x0;
    return x0;
}

/* ------------------------------------------------------------------------ */
/* Exact enumeration of the sector (tiny lattices only)                      */
/* ------------------------------------------------------------------------ */

static int next_combination(int* c, int k, int n)
{
    int i = k - 1;
    while (i >= 0 && c[i] == n - k + i) --i;
    if (i < 0) return 0;
    c[i]++;
    for (int j = i + 1; j < k; ++j) c[j] = c[j - 1] + 1;
    return 1;
}

/* Number of configurations with n_up up and n_dn down electrons. */
int64_t orc_sector_size(const orc_problem* P)
{
    double a = 1, b = 1;
    for (int i = 0; i < P->n_up; ++i) a = a * (P->n_sites - i) / (i + 1);
    for (int i = 0; i < P->n_dn; ++i) b = b * (P->n_sites - i) / (i + 1);
    return (int64_t)llround(a * b);
}

/* List every sector configuration (ascending occupied lists, up choice
 * outer, down choice inner, each in lexicographic order). */
int64_t orc_enumerate(const orc_problem* P, uint8_t* occ_out)
{
    int nu = P->n_up, nd = P->n_dn, ns = P->n_sites, N = nu + nd;
    int cu[64], cd[64];
    int64_t cnt = 0;
    for (int i = 0; i < nu; ++i) cu[i] = i;
    do {
        for (int i = 0; i < nd; ++i) cd[i] = i;
        do {
            for (int i = 0; i < nu; ++i) occ_out[cnt * N + i] = (uint8_t)cu[i];
            for (int i = 0; i < nd; ++i) occ_out[cnt * N + nu + i] = (uint8_t)(ns + cd[i]);
            ++cnt;
        } while (nd > 0 && next_combination(cd, nd, ns));
    } while (nu > 0 && next_combination(cu, nu, ns));
    return cnt;
}

/* Exact |Psi_n|^2 / <Psi|Psi> over the whole sector, from log amplitudes. */
void orc_exact_weights(const orc_problem* P, int64_t n_conf, const uint8_t* occ, double* w)
{
    int N = P->n_up + P->n_dn;
    double mx = -INFINITY;
    double* la = (double*)malloc(sizeof(double) * n_conf);
    for (int64_t i = 0; i < n_conf; ++i) {
        int s;
        orc_log_psi(P, occ + i * N, &la[i], &s);
        if (s == 0) la[i] = -INFINITY;
        if (la[i] > mx) mx = la[i];
    }
    double tot = 0.0;
    for (int64_t i = 0; i < n_conf; ++i) { w[i] = exp(2.0 * (la[i] - mx)); tot += w[i]; }
    for (int64_t i = 0; i < n_conf; ++i) w[i] /= tot;
    free(la);
}

/* ------------------------------------------------------------------------ */
/* Accelerated linear method (Sec. II.B)                                     */
/* ------------------------------------------------------------------------ */

/* Products of the linear method's matrices with x = (x_0, x_1 .. x_nv) over
 * the basis {Psi, Psi^1 .. Psi^nv}, Psi^j = dPsi/dalpha_j (component 0 is
 * Psi itself, O_0 = 1):
 *   Hx_i = sum_n w_n sum_{pq} Q_{n q p i} sum_mu L^mu_pq sum_{rs} R^mu_rs sum_j Q_{n r s j} x_j
 *          + c0 Sx_i                                                  (Eq. 10)
 *   Sx_i = sum_n w_n O_i(n) sum_j O_j(n) x_j,
 * with Q_{n r s j} = <n| a+_r a_s |Psi^j> / Psi_n (Eq. 10) and the
 * Hamiltonian in the factored form of Eq. 9, H = c0 + sum_mu Lhat_mu Rhat_mu,
 * Lhat_mu = sum_{ij} L^mu_ij sum_sigma a+_{i sigma} a_{j sigma} (spatial
 * matrices L^mu, R^mu of n_sites^2 entries).  w_n = 1/n_s when wgt is NULL.
 * Every Q is built from scratch: the configuration n' with
 * <n| a+_r a_s |n'> != 0, its explicit Jordan-Wigner sign, a fresh amplitude
 * Psi_n' and a fresh O(n') (so Psi^j_n' = Psi_n' O_j(n')).  Sx may be NULL.
 * Returns -1 if a pairing submatrix is singular. */
int orc_lm_apply(const orc_problem* P, int64_t n_s, const uint8_t* occ, const double* wgt,
                 int n_mu, const double* Lf, const double* Rf, double c0, const double* x,
                 double* Hx, double* Sx)
{
    const int M = n_orb_M(P), N = P->n_up + P->n_dn, ns = P->n_sites;
    const int64_t nv = orc_n_params(P);
    memset(Hx, 0, sizeof(double) * (nv + 1));
    if (Sx) memset(Sx, 0, sizeof(double) * (nv + 1));
    /* per sample: every (r, s) of one spin with <n| a+_r a_s |n'> != 0
     * (r occupied, s = r or empty: at most ns per electron) */
    const int nmax = N * ns;
    double* ratio = (double*)malloc(sizeof(double) * nmax);
    double* Op = (double*)malloc(sizeof(double) * (size_t)nmax * nv);   /* O(n') rows */
    int* er = (int*)malloc(sizeof(int) * nmax);
    int* es = (int*)malloc(sizeof(int) * nmax);
    double* On = (double*)malloc(sizeof(double) * nv);
    double* w = (double*)malloc(sizeof(double) * (n_mu > 0 ? n_mu : 1));
    uint8_t bits[512], bnp[512], tmp[512], occp[256];
    int rc = 0;
    for (int64_t n = 0; n < n_s && rc == 0; ++n) {
        const uint8_t* o = occ + n * N;
        const double wn = wgt ? wgt[n] : 1.0 / (double)n_s;
        occ_to_bits(P, o, bits);
        double la0;
        int s0;
        orc_log_psi(P, o, &la0, &s0);
        if (s0 == 0 || orc_logderiv(P, o, On) != 0) { rc = -1; break; }
        int ne = 0;
        for (int r = 0; r < M; ++r) {
            if (!bits[r]) continue;
            const int lo = r < ns ? 0 : ns;
            for (int s = lo; s < lo + ns; ++s) {
                if (s != r && bits[s]) continue;
                /* n' = n with the electron at r moved to s */
                memcpy(bnp, bits, M);
                bnp[r] = 0;
                bnp[s] = 1;
                const int sg = hop_sign(M, bnp, r, s, tmp);      /* a+_r a_s |n'> = sg |n> */
                bits_to_occ(M, bnp, occp);
                double* row = Op + (size_t)ne * nv;
                if (orc_logderiv(P, occp, row) != 0) { rc = -1; break; }
                ratio[ne] = (double)sg * amp_ratio(P, occp, la0, s0);
                er[ne] = r;
                es[ne] = s;
                ++ne;
            }
            if (rc) break;
        }
        if (rc) break;
        /* y_rs = sum_j Q_{n r s j} x_j, w_mu = sum_rs R^mu_rs y_rs */
        for (int mu = 0; mu < n_mu; ++mu) w[mu] = 0.0;
        for (int e = 0; e < ne; ++e) {
            double ox = x[0];
            const double* row = Op + (size_t)e * nv;
            for (int64_t j = 0; j < nv; ++j) ox += row[j] * x[1 + j];
            const double y = ratio[e] * ox;
            const int i = er[e] % ns, k = es[e] % ns;
            for (int mu = 0; mu < n_mu; ++mu) w[mu] += Rf[((size_t)mu * ns + i) * ns + k] * y;
        }
        /* z_pq = sum_mu L^mu_pq w_mu; Hx_i += w_n sum_{pq} z_pq Q_{n q p i}:
         * the excitation of Q_{n q p i} moves the electron at q to p, i.e.
         * entry e with (er, es) = (q, p) */
        for (int e = 0; e < ne; ++e) {
            const int q = er[e] % ns, p = es[e] % ns;
            double z = 0.0;
            for (int mu = 0; mu < n_mu; ++mu) z += Lf[((size_t)mu * ns + p) * ns + q] * w[mu];
            const double c = wn * z * ratio[e];
            if (c == 0.0) continue;
            const double* row = Op + (size_t)e * nv;
            Hx[0] += c;
            for (int64_t i = 0; i < nv; ++i) Hx[1 + i] += c * row[i];
        }
        /* overlap and the constant c0 */
        double ox = x[0];
        for (int64_t j = 0; j < nv; ++j) ox += On[j] * x[1 + j];
        Hx[0] += wn * c0 * ox;
        for (int64_t i = 0; i < nv; ++i) Hx[1 + i] += wn * c0 * ox * On[i];
        if (Sx) {
            Sx[0] += wn * ox;
            for (int64_t i = 0; i < nv; ++i) Sx[1 + i] += wn * ox * On[i];
        }
    }
    free(ratio); free(Op); free(er); free(es); free(On); free(w);
    return rc;
}

/* Annihilation / creation on a determinant given as occupation bits (for the
 * operator-matrix checks of the factored Hamiltonian): returns the sign and
 * rewrites bits, 0 if the result vanishes. */
int orc_apply_hop(int M, const uint8_t* bits, int p, int q, uint8_t* out)
{
    return hop_sign(M, bits, p, q, out);
}

/* Number of OpenMP threads of the oracle's parallel loops (the CPU baseline
 * is timed on all host cores and on one). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
