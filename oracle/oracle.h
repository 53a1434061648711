/*
 * Plain FP64 CPU oracle for the matrix-free SR hot path (arXiv:1108.0900).
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the package smoke check and
 * the benchmark's CPU-baseline leg; never by the product path.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

typedef struct orc_problem {
    int n_sites;            /* spatial orbitals; M = 2 n_sites spin orbitals  */
    int n_up, n_dn;         /* fixed sector (Sec. III)                         */
    int ham;                /* 0 Hubbard, 1 ab initio                          */
    int n_bonds;            /* Hubbard bond list (i, j) and hopping t          */
    const int32_t* bonds;
    const double* bond_t;
    double U;
    int n_chol;             /* ab initio: h[n][n], L[n_chol][n][n]             */
    const double* h;
    const double* chol;
    int n_corr;             /* correlators: sites corr_sites[corr_ptr[c]..]    */
    const int32_t* corr_ptr;
    const int32_t* corr_sites;
    const int32_t* corr_class; /* class of every correlator (NULL: each its own);
                               correlators of one class share one parameter
                               block (translation-invariant correlators)     */
    const double* C;        /* correlator amplitudes, class-major              */
    const double* f;        /* pairing f_pq, p < q, row-major upper triangle    */
} orc_problem;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_pfaffian(int n, double* A, double* logabs, int* sign);
int orc_inverse(int n, const double* A, double* X);
int64_t orc_n_corr_params(const orc_problem* P);
int64_t orc_n_params(const orc_problem* P);
int64_t orc_corr_state(const orc_problem* P, const uint8_t* occ, int c);
void orc_log_psi(const orc_problem* P, const uint8_t* occ, double* logabs, int* sign);
int orc_logderiv(const orc_problem* P, const uint8_t* occ, double* O);
double orc_hamiltonian_element(const orc_problem* P, const uint8_t* occ_n, const uint8_t* occ_np);
double orc_local_energy_hubbard(const orc_problem* P, const uint8_t* occ);
double orc_local_energy_abinitio(const orc_problem* P, const uint8_t* occ);
double orc_local_energy_abinitio_bruteforce(const orc_problem* P, const uint8_t* occ);
double orc_local_energy(const orc_problem* P, const uint8_t* occ);
int orc_sample(const orc_problem* P, int n_walkers, uint8_t* occ, uint64_t* step, uint64_t seed,
               int n_burn, int n_spw, uint8_t* out_occ, double* min_margin, int64_t* accepts,
               double close_tol, int64_t* first_close);
int orc_measure(const orc_problem* P, int64_t n_s, const uint8_t* occ, double* E, double* O);
void orc_mean_O(int64_t n_s, int64_t nv, const double* O, double* Obar);
void orc_gradient(int64_t n_s, int64_t nv, const double* O, const double* E, double* g,
                  double* E_mean);
void orc_dense_S(int64_t n_s, int64_t nv, const double* O, double* S);
void orc_apply_S(int64_t n_s, int64_t nv, const double* O, const double* Obar, const double* v,
                 double eps, double* out);
/* Eq. 7 from compact rows (ascending occupation, correlator states, the
 * values of the nonzero pairing derivatives with their position pairs), for
 * k vectors [k][nv]; Obar_out[nv] = mean of the rows.  See oracle.c. */
void orc_apply_S_compact(const orc_problem* P, int64_t n_s, const uint8_t* occ, const int64_t* cs, int n_pair,
                         const int32_t* pairs, const double* pf, int k, const double* v, double eps,
                         double* out, double* Obar_out);
int orc_cg(int64_t n_s, int64_t nv, const double* O, const double* g, double eps, double tol,
           int max_iter, double* x, int* iters, double* true_rel_res);
/* SR parameter update (Sec. II.A, after Eq. 2): x = -tau y, x_0 = 1 - tau E_mean - Obar . x,
 * alpha_out = alpha + x / x_0.  Returns x_0. */
double orc_sr_update(int64_t nv, const double* alpha, const double* y, double tau, double E_mean,
                     const double* Obar, double* alpha_out);
int64_t orc_sector_size(const orc_problem* P);
int64_t orc_enumerate(const orc_problem* P, uint8_t* occ_out);
void orc_exact_weights(const orc_problem* P, int64_t n_conf, const uint8_t* occ, double* w);
/* Linear method (Sec. II.B): Hx and Sx over the basis {Psi, Psi^1 .. Psi^nv}
 * by Eq. 10 with the factored Hamiltonian of Eq. 9 (spatial L^mu, R^mu,
 * [n_mu][n_sites][n_sites], plus the constant c0); wgt NULL = 1/n_s. */
int orc_lm_apply(const orc_problem* P, int64_t n_s, const uint8_t* occ, const double* wgt,
                 int n_mu, const double* Lf, const double* Rf, double c0, const double* x,
                 double* Hx, double* Sx);
int orc_apply_hop(int M, const uint8_t* bits, int p, int q, uint8_t* out);

void orc_set_threads(int n);

#endif
