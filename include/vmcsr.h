/*
 * vmcsr — GB300-native matrix-free stochastic reconfiguration (SR) for a
 * correlator-product-state (CPS) x pfaffian wavefunction.
 *
 * The method is that of Neuscamman, Umrigar and Chan, "Optimizing large
 * parameter sets in variational quantum Monte Carlo" (arXiv:1108.0900):
 *   Sec. II.A, Eq. 2   the SR linear system <Psi^i|(1 - tau H)|Psi> = sum_j S_ij x_j;
 *   Sec. II.A, Eq. 3   derivative ratios Psi^i_n / Psi_n sampled from |Psi_n|^2;
 *   Sec. II.A, Eq. 7   S z evaluated by interchanging the sums, O(n_s n_v);
 *   Sec. II.A          conjugate gradient instead of building S;
 *   Sec. II.C, Eq. 11  |Psi> = prod_p C_p (sum_{i<j} f_ij a+_i a+_j)^{N/2} |0>;
 *   Sec. III           sampling restricted to fixed N and S_z.
 *
 * Conventions shared by every entry point
 *   - M = 2 n_sites spin orbitals; spin orbital p = sigma * n_sites + site.
 *   - Parameter vector alpha (length n_v): correlator amplitudes first
 *     (correlator c occupies 4^{m_c} consecutive entries, m_c = its site
 *     count, local state idx_c = sum_j 4^j (n_{s_j up} + 2 n_{s_j dn})),
 *     then the pairing amplitudes f_pq, p < q, in row-major upper-triangle
 *     order (M(M-1)/2 entries).
 *   - O_k(n) = (dPsi_n / dalpha_k) / Psi_n.  Eliminating x_0 from Eq. 2 with
 *     O_0 = 1 gives S x = -tau g with the covariance S_ij = <O_i O_j> -
 *     <O_i><O_j> and g_i = <E_L O_i> - <E_L><O_i>; every mean uses weight 1/n_s.
 *     The library solves (S + shift I) y = g and returns y.
 *   - Sample s = walker * samples_per_walker + j.
 *   - Every function returns VMC_OK (0) or a negative VMC_ERR_* code; no
 *     exception crosses this boundary.  Pointers marked "host" are read or
 *     written synchronously; pointers marked "device" are CUDA device
 *     addresses on the handle's device and are only touched by work enqueued
 *     on `stream` (a cudaStream_t passed as void*, NULL = legacy stream).
 *   - The caller owns every pointer it passes; the handle owns its walker
 *     state, its O store and all scratch buffers.
 */
#ifndef VMCSR_H
#define VMCSR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VMC_OK 0
#define VMC_ERR_INVALID_ARG -1
#define VMC_ERR_OOM -2
#define VMC_ERR_SINGULAR -3
#define VMC_ERR_NONFINITE -4
#define VMC_ERR_NOT_CONVERGED -5
#define VMC_ERR_TIMEOUT -6
#define VMC_ERR_CUDA -7
#define VMC_ERR_UNSUPPORTED -8
#define VMC_ERR_STATE -9

#define VMC_HUBBARD 0
#define VMC_ABINITIO 1

/* arithmetic of the walkers (sampling, local energy, derivative ratios) */
#define VMC_FP64 0      /* every walker quantity in FP64                         */
#define VMC_FP32 1      /* FP32 ratios and inverse updates, FP64 sums             */

/* O-store / S-product precisions */
#define VMC_STORE_FP64 0  /* FP64 storage, FP64 arithmetic                        */
#define VMC_STORE_FP32 1  /* FP32 storage, FP64 accumulation                      */
#define VMC_STORE_BF16 2  /* BF16 storage, FP32 accumulation                      */
#define VMC_STORE_FP32_F32ACC 3  /* FP32 storage, FP32 accumulation               */

/* CG modes */
#define VMC_CG_FP64 0   /* plain CG, FP64 vectors and FP64 S products             */
#define VMC_CG_MIXED 1  /* BF16-stream inner CG (FP32 vectors, FP64 scalars),
                           refined against the FP32 store with FP64 accumulation  */
#define VMC_CG_FP32 2   /* like MIXED but the inner product streams FP32          */
#define VMC_CG_BLOCK4 3 /* like MIXED with an enlarged block CG as the inner solve:
                           the right-hand side split into four parameter-group
                           columns (first / second half of the correlators,
                           same-spin / opposite-spin pairing), one four-vector
                           BF16 product per inner iteration, solution = column
                           sum; needs >= 2 correlators (else UNSUPPORTED)       */
#define VMC_CG_MIXED64 4 /* like MIXED, but the flexible outer iteration and the
                           reported true residual use the FP64 store (needs
                           keep_fp64_store; pass g from sr_gradient over the FP64
                           store): the residual is against the FP64 operator    */

typedef struct vmc_ctx* vmc_handle;

/* Lattice: n_sites spatial orbitals (<= 64) and, for the Hubbard model, the
 * bond list (bonds[2b], bonds[2b+1]) with hopping bond_t[b]; a repeated bond
 * adds its hopping again.  Arrays are host pointers, copied by vmc_create. */
typedef struct {
    int n_sites;
    int n_bonds;
    const int32_t* bonds;
    const double* bond_t;
} vmc_lattice;

/* Hamiltonian.  VMC_HUBBARD: H = -sum_b t_b sum_s (c+_is c_js + h.c.)
 * + U sum_i n_i,up n_i,dn.  VMC_ABINITIO: H = sum_{pq,s} h_pq a+_ps a_qs
 * + 1/2 sum_{pqrs,st} (pq|rs) a+_ps a+_rt a_st a_qs with
 * (pq|rs) = sum_mu L^mu_pq L^mu_rs (the factorised form of Eq. 9 with R = L);
 * h is [n_sites][n_sites] and chol is [n_chol][n_sites][n_sites], host. */
typedef struct {
    int kind;
    double U;
    int n_chol;
    const double* h;
    const double* chol;
} vmc_hamiltonian;

/* Ansatz (Eq. 11): sector (n_up, n_dn) with n_up + n_dn even and <= 64, and
 * correlator site lists corr_sites[corr_ptr[c] .. corr_ptr[c+1]) (each <= 9
 * sites, host arrays).  The pairing runs over all spin orbitals.
 * corr_class[n_corr] (host, may be NULL = every correlator its own class)
 * lets correlators share parameters: the correlators of one class (the
 * translates of one correlator, as in Sec. III.A's translationally invariant
 * 3x3 correlators) read one block of 4^m amplitudes, so O of a shared
 * amplitude sums over them.  Classes are numbered 0 .. n_class-1, all used,
 * with one site count per class; the parameter blocks follow class order. */
typedef struct {
    int n_up;
    int n_dn;
    int n_corr;
    const int32_t* corr_ptr;
    const int32_t* corr_sites;
    const int32_t* corr_class;
} vmc_ansatz;

typedef struct {
    int n_walkers;          /* Markov chains                                       */
    int samples_per_walker; /* samples stored per vmc_sample call                  */
    int walker_precision;   /* VMC_FP64 or VMC_FP32                                 */
    int keep_fp64_store;    /* 1: keep an FP64 O store (needed by VMC_CG_FP64)       */
    int keep_lowp_store;    /* 1: keep FP32 + BF16 O stores (needed by MIXED/FP32)   */
    int refresh_every;      /* sweeps between from-scratch rebuilds of each walker's
                               pairing inverse during vmc_sample (0: only at the start
                               of each call); bounds the drift of the rank-2 updates   */
    int fp64_refresh;       /* FP32 walkers only, 1: after the chains have run, every
                               stored sample's pairing inverse, log-amplitude, E_L and
                               O are evaluated from scratch in FP64 and the stores are
                               written from those values (FP32 / BF16 rounding of FP64
                               results); the chains' own E_L is kept for
                               vmc_sample_stats                                        */
} vmc_options;

typedef struct {
    int iterations;          /* S products in the inner (or only) Krylov loop      */
    int refinements;         /* outer refinement steps (mixed modes)                */
    int residual_products;   /* high-precision residual products (mixed modes)      */
    int converged;           /* 1 if the true residual met tol                      */
    double true_rel_residual;/* |g - (S + shift I) x| / |g|, FP64 accumulation over
                                the mode's reference store (FP64 or FP32)           */
} vmc_cg_info;

/* Create a handle on the current CUDA device.  Copies every input.  Errors:
 * INVALID_ARG (sizes out of range, odd N, > 64 sites, bad bond or site index),
 * OOM, CUDA. */
int vmc_create(const vmc_lattice* lat, const vmc_hamiltonian* ham, const vmc_ansatz* ans,
               const vmc_options* opt, vmc_handle* out);
int vmc_destroy(vmc_handle h);

/* Number of variational parameters n_v and of correlator parameters. */
int vmc_num_params(vmc_handle h, int64_t* n_v, int64_t* n_corr_params);

/* Set the correlator amplitudes C[n_corr_params] and pairing f[M(M-1)/2]
 * (host, FP64, layout above).  Waits for all work queued on the device (any
 * stream) before it overwrites the parameters.  Errors: SINGULAR if some C is
 * zero. */
int vmc_set_params(vmc_handle h, const double* C, const double* f);

/* Read the current parameters back (host C[n_corr_params], f[M(M-1)/2],
 * FP64, the layout of vmc_set_params); either pointer may be NULL. */
int vmc_get_params(vmc_handle h, double* C, double* f, void* stream);

/* Set walker configurations: occ[n_walkers][N] ascending occupied spin
 * orbitals (host, uint8) with n_up orbitals below n_sites; step[n_walkers]
 * (host, may be NULL = 0) is each chain's proposal counter.  Waits for all
 * work queued on the device (any stream) before it overwrites the walkers.
 * Errors: INVALID_ARG for a configuration outside the sector. */
int vmc_set_walkers(vmc_handle h, const uint8_t* occ, const uint64_t* step);
/* Read back walker configurations (ascending) and counters (host, may be
 * NULL) once the work queued on `stream` is done; a sampling call queued on
 * another stream must be waited for by the caller. */
int vmc_get_walkers(vmc_handle h, uint8_t* occ, uint64_t* step, void* stream);

/* Metropolis sampling from |Psi_n|^2 in the fixed sector (Sec. II.A, Sec. III).
 * Each walker first rebuilds its pairing inverse from scratch, runs n_burn
 * sweeps, then samples_per_walker sweeps each ending in a stored sample; a
 * sweep is N proposals.  A proposal moves the a-th occupied orbital
 * (ascending) to the k-th empty orbital of the same spin (ascending); a, k
 * and u come from Philox4x32-10 with key (seed lo, seed hi) and counter
 * (walker, step lo, step hi, 0): a = hi32(r0 N), k = hi32(r1 n_empty),
 * u = (r2 >> 8) 2^-24, accepted iff u < |Psi'/Psi|^2.  At each stored sample
 * the walker writes E_L, its ascending occupation, the correlator states and
 * the pairing block of O into the handle's O store.  Errors: SINGULAR (a
 * walker's pairing submatrix could not be inverted), NONFINITE, CUDA. */
int vmc_sample(vmc_handle h, int n_burn, uint64_t seed, void* stream);

/* Health of the last vmc_sample (no counterpart in the paper).  Every chain
 * sums ln|Psi'/Psi| over its accepted moves (FP64 sum of its ratios); for the
 * stored samples j > 0 of walker w this running change is compared with the
 * change of ln|Psi| evaluated from scratch in FP64 (vmc_logpsi):
 *   drift = |(run_j - run_0) - (lnPsi_j - lnPsi_0)|,
 * which measures the accumulated error of the rank-2 inverse updates and
 * ratios.  With fp64_refresh, el_refresh_change is |E_L(chain) -
 * E_L(FP64 refresh)| / max(1, |E_L(FP64 refresh)|) per sample.  Needs the
 * samples of a vmc_sample call (n_walkers x samples_per_walker).  Errors:
 * STATE. */
typedef struct {
    double lnpsi_drift_max;
    double lnpsi_drift_mean;
    int refreshed;                 /* 1 if the stored samples come from an FP64 refresh */
    double el_refresh_change_max;
    double el_refresh_change_mean;
} vmc_sample_stats_t;
int vmc_sample_stats(vmc_handle h, vmc_sample_stats_t* out, void* stream);

/* Several lattices of uneven size in one launch (no counterpart in the
 * paper, which states the method per problem).  vmc_sample_batch does
 * vmc_sample(hs[b], n_burn, seeds[b]) for b < n (n <= 16 distinct handles of
 * one device and one walker precision) as a single kernel launch: each warp
 * finds its problem from the running sum of the walker counts, and every warp
 * gets the shared-memory slice of the largest problem.  Each handle then holds
 * exactly the samples its own vmc_sample with the same seed gives.  hs and
 * seeds are host arrays.  Synchronizes `stream`.  Errors: INVALID_ARG (n out
 * of range, a repeated handle, mixed precisions or devices), STATE, and the
 * errors of vmc_sample. */
int vmc_sample_batch(const vmc_handle* hs, int n, int n_burn, const uint64_t* seeds, void* stream);

/* out[b] = (S_b + shift I) V[b] (Eq. 7 with the covariance term) for every
 * handle b < n, each over its own samples: one streaming launch reads every
 * handle's store (the generic per-sample pass; its CTAs are split among the
 * problems in proportion to their stored bytes), then each handle's
 * correlator sums and finish run.  V and out are host arrays of n device
 * pointers to FP64 vectors of the handle's n_v; store is VMC_STORE_FP64 or
 * VMC_STORE_FP32 (FP64 accumulation).  Synchronizes `stream`.  Errors:
 * INVALID_ARG, STATE, UNSUPPORTED (a pairing block beyond shared memory). */
int sr_apply_S_batch(const vmc_handle* hs, int n, const double* const* V, double* const* out, double shift,
                     int store, void* stream);

/* Evaluate E_L and O for caller-given configurations occ[n_s][N] (host,
 * ascending, n_s <= n_walkers * samples_per_walker), recomputing each
 * pairing inverse from scratch; the result replaces the O store and the
 * handle then holds n_s samples. */
int vmc_measure(vmc_handle h, const uint8_t* occ, int64_t n_s, void* stream);

/* Number of samples currently in the O store. */
int vmc_num_samples(vmc_handle h, int64_t* n_s);

/* Copy the O store out (host pointers, each may be NULL): occ[n_s][N],
 * E_L[n_s], corr_state[n_s][n_corr] (uint32), pf[n_s][P] with
 * P = n_up(n_up-1)/2 + n_dn(n_dn-1)/2 + n_up n_dn in block order
 * (up-up triangle row-major, down-down triangle, up-down rectangle
 * row-major over ascending positions) converted to FP64 from the store
 * `store` (VMC_STORE_*).  Element (a, b), a < b, is O of f_{occ[a] occ[b]}. */
int vmc_get_samples(vmc_handle h, uint8_t* occ, double* E_L, uint32_t* corr_state, double* pf,
                    int store, void* stream);

/* ln|Psi_n| for every stored sample (device out[n_s], FP64 pfaffian from scratch). */
int vmc_logpsi(vmc_handle h, double* out, void* stream);
/* Adjoint of ln|Psi_n| with respect to alpha (Eq. 3's ratios): with w
 * (device [n_s] FP64) writes grad[k] = sum_s w_s O_k(n_s) (device [n_v]),
 * recomputing every pairing inverse from scratch in FP64 instead of reading
 * the store; with w == NULL it instead rewrites the O store from scratch
 * (grad unused). */
int vmc_logpsi_backward(vmc_handle h, const double* w, double* grad, void* stream);

/* Sample means and the SR right-hand side (Eq. 2 after eliminating x_0):
 * Obar (kept in the handle), E_mean = <E_L>, g = <E_L O> - <E_L> Obar
 * (device g[n_v]), FP64 accumulation over the store of `store`
 * (VMC_STORE_FP64 or VMC_STORE_FP32).  e_stats (host, may be NULL) receives
 * {E_mean, E_variance, standard error over walkers}. */
int sr_gradient(vmc_handle h, double* g, double* e_stats, int store, void* stream);

/* out = (S + shift I) V for k right-hand sides (Eq. 7 with the covariance
 * term): V and out are device [k][n_v] FP64 (column j at offset j n_v),
 * 1 <= k <= 4; `store` picks the O store and arithmetic (VMC_STORE_*).
 * sr_gradient must have run since the last sampling call (it sets Obar).
 * Synchronizes `stream` to read the kernels' status (TIMEOUT, see
 * vmc_set_wait_limit). */
int sr_apply_S(vmc_handle h, const double* V, double* out, int k, double shift, int store,
               void* stream);

/* Solve (S + shift I) x = g (device g, x [n_v] FP64) by conjugate gradient
 * (Sec. II.A), x_0 = 0, until the true relative residual is <= tol or
 * max_iter products; mode VMC_CG_*.  info (host) is filled. */
int sr_cg_solve(vmc_handle h, const double* g, double shift, double tol, int max_iter, int mode,
                double* x, vmc_cg_info* info, void* stream);

/* Inner tolerance of the mixed solves (no counterpart in the paper): each
 * flexible outer step asks the low-precision inner CG for a relative
 * residual of max(floor, half of what the outer iteration still needs);
 * floor 0 restores the default (0.1 for the BF16 inner solves, 1e-3 for
 * VMC_CG_FP32).  Errors: INVALID_ARG unless 0 <= floor < 1. */
int sr_set_inner_tol(vmc_handle h, double floor);

/* SR parameter update (Sec. II.A): after the solve of Eq. 2 with x_0
 * eliminated, (S + shift I) y = g, the coefficients of the projected state
 * (1 - tau H)|Psi> are x = -tau y and x_0 = 1 - tau <E_L> - Obar . x, and
 * every parameter moves to alpha_k + x_k / x_0 on the device (the FP32
 * copies, 1/C and the antisymmetric F matrices follow).  y is device [n_v]
 * FP64; <E_L> and Obar are those of the last sr_gradient over `store`
 * (VMC_STORE_FP64, VMC_STORE_FP32 or VMC_STORE_BF16).  x0 (host, may be
 * NULL) receives x_0.  The stored samples then belong to the old
 * parameters: sample again before the next gradient.  Errors: STATE when no
 * gradient was taken over `store`; NONFINITE when x_0 <= 0 or not finite (tau
 * beyond the first-order projector; nothing is changed), or when an updated
 * parameter is not finite; SINGULAR when an updated C is zero. */
int sr_update(vmc_handle h, const double* y, double tau, int store, double* x0, void* stream);

/* Rank-local sums for a solve whose samples are spread over several processes
 * (the paper distributes the samples over processors, Sec. II.A): a sum
 * all-reduce of these over the ranks gives the global moments and products.
 * sr_local_moments: sumO = sum_s O_s and sumEO = sum_s E_L(s) O_s (device
 * [n_v] FP64), scal = {sum_s E_L(s), n_s} (host), FP64 accumulation over
 * `store`; it also leaves this rank's own Obar in the handle.
 * sr_local_product: out = sum_s (O_s . v) O_s over this rank's samples
 * (device v, out [n_v] FP64; FP64 accumulation over the FP64 or FP32 store;
 * sr_local_moments or sr_gradient must have run over that store).  The global
 * (S + shift I) v is then (sum over ranks of out) / N - Obar (Obar . v) +
 * shift v with the global N and Obar.  Errors: STATE without samples or
 * moments. */
int sr_local_moments(vmc_handle h, double* sumO, double* sumEO, double* scal, int store, void* stream);
int sr_local_product(vmc_handle h, const double* v, double* out, int store, void* stream);

/* Accelerated linear method (Sec. II.B).  The products with x = (x_0, x_1 ..
 * x_nv) of the matrices of Eq. 8 over the basis {Psi, Psi^1 .. Psi^nv}
 * (Psi^j = dPsi/dalpha_j; component 0 is Psi itself), estimated from the
 * stored samples by Eq. 10:
 *   Hx_i = (1/n_s) sum_n sum_pq Q_{n q p i} sum_mu L^mu_pq sum_rs R^mu_rs
 *          sum_j Q_{n r s j} x_j + c0 Sx_i,   Q_{n r s j} = <n|a+_r a_s|Psi^j>/Psi_n,
 *   Sx_i = (1/n_s) sum_n O_i(n) sum_j O_j(n) x_j   (O_0 = 1),
 * with the Hamiltonian written in the factored form of Eq. 9,
 * H = c0 + sum_mu Lhat_mu Rhat_mu over spin-summed one-body operators
 * Lhat = sum_ij L_ij sum_s a+_is a_js.  The handle builds the factors from
 * its Hamiltonian: a one-body term K enters as (K Nhat + Nhat K) / 2N (exact
 * at fixed N; this split makes the sampled H symmetric); Hubbard U as
 * (U/2) E_ii E_ii per site with c0 = -U N / 2; the ab initio two-body part
 * as the pairs (L^mu, L^mu)/sqrt(2) with h - J/2, J_ps = sum_q (pq|qs).
 * x, Hx, Sx: device [n_v + 1] FP64 (Sx may be NULL); Hx and Sx are
 * overwritten.  store: VMC_STORE_FP64 (FP64 arithmetic) or VMC_STORE_FP32
 * (FP32 arithmetic, FP64 accumulation into Hx / Sx) over the samples of the
 * last vmc_sample / vmc_measure.  Errors: INVALID_ARG, STATE (no samples,
 * no parameters, store not kept), UNSUPPORTED (the per-sample workspace of
 * (2N + 3(M - N))(N + 1) + n_sites^2 + n_mu values exceeds shared memory),
 * OOM, CUDA. */
int lm_apply(vmc_handle h, const double* x, double* Hx, double* Sx, int store, void* stream);

typedef struct {
    int iterations;          /* Davidson steps (one lm_apply each)                  */
    int restarts;            /* basis restarts                                      */
    int converged;           /* 1 if the relative residual met tol                  */
    double eigenvalue;       /* lowest eigenvalue theta of the shifted Eq. 8         */
    double rel_residual;     /* |(H + aD) u - theta (S + eps D) u| / |theta (S + eps D) u| */
    double Sx0;              /* (S x)_0 = x_0 + sum_j Obar_j x_j of the returned x   */
} vmc_lm_info;

/* Lowest eigenpair of Eq. 8 with diagonal shifts on the parameter block,
 * (H + shift_H D) x = theta (S + shift_S D) x, D = diag(0, 1, .., 1), by the
 * generalized Davidson method (Sec. II.B; Morgan's method: Rayleigh-Ritz on
 * an orthonormal basis grown by the preconditioned residual
 * -r / diag(S + shift_S D); at max_sub columns the basis restarts from the
 * current and the previous Ritz vectors), every product through lm_apply,
 * starting from x = e_0 (the current wavefunction).  Returns x (device
 * [n_v + 1] FP64) scaled to x_0 = 1.  shift_S > 0 keeps S + shift_S D
 * positive definite.  The projected problem (at most max_sub = 3..64
 * columns) is solved on the host.  Errors: INVALID_ARG, STATE (as
 * lm_apply), NOT_CONVERGED (max_iter reached; x and info hold the last Ritz
 * pair), NONFINITE, OOM, CUDA. */
int lm_solve(vmc_handle h, double shift_H, double shift_S, double tol, int max_iter, int max_sub, double* x,
             vmc_lm_info* info, int store, void* stream);

/* Linear-method parameter update (Sec. II.B): alpha_k += x_k / Sx0 with Sx0
 * = (S x)_0 from lm_solve (the new state's component along Psi once the
 * basis is orthogonalised to Psi).  x: device [n_v + 1].  The stored samples
 * are then stale.  Errors: INVALID_ARG (Sx0 zero or not finite), STATE,
 * SINGULAR (a correlator amplitude became 0), NONFINITE, CUDA. */
int lm_update(vmc_handle h, const double* x, double Sx0, void* stream);

/* Measurement support (no counterpart in the paper).  vmc_profile(h, 1)
 * resets the counters and starts recording: every kernel the handle launches
 * is counted, and each launch of the O-store streaming kernel (the Eq. 7
 * gather/scatter pass and the gradient pass) is bracketed by CUDA events on
 * its stream.  vmc_profile(h, 0) stops recording.  Recording adds two event
 * records per streaming launch and nothing else. */
int vmc_profile(vmc_handle h, int enable);
/* Totals since the last vmc_profile(h, 1) (host outputs, each may be NULL):
 * launches_all = kernels launched; for streaming launches over the store
 * `store` (VMC_STORE_*; FP32 with FP64 and with FP32 accumulation are
 * counted apart) their number, summed device time in ms and algorithmic
 * bytes = n_s (2 n_corr + N + P * element size) per launch (the O store read
 * once).  Waits for the recorded events. */
int vmc_profile_read(vmc_handle h, int store, int64_t* launches_all, int64_t* pass_launches, double* pass_ms,
                     double* pass_bytes);

/* Allocation-free pairing-block product (no counterpart in the paper).
 * For callers that cannot call cudaMalloc: code running inside a memory budget
 * that a pool allocator already owns (a fresh cudaMalloc would fail) and
 * latency-critical loops (cudaMalloc / cudaFree synchronise the device).  No
 * handle is needed and nothing is allocated: the caller passes every input and
 * output as device pointers, and the scratch (one partial image of the pairing
 * block per CTA) is a fixed device array of 128 x 8128 floats (4.2 MB) that
 * every GPU which loads the library holds until the process exits.
 *   occ  [n_s][occ_stride] uint8, ascending occupied spin orbitals (n_up below
 *        n_sites, then n_dn), pf [n_s][pf_stride] FP32 pairing blocks in the
 *        block order of vmc_get_samples, v [M(M-1)/2] FP32 (f_pq order);
 *   t    [n_s] FP32 out: t_s = sum_e pf_s[e] v[pq(e)];
 *   out  [M(M-1)/2] FP64 out: out[pq] = sum_s t_s pf_s[e] at pq(e) (FP32
 *        accumulation per CTA, FP64 across CTAs).
 * This is the pairing-block half of the Eq. 7 product without the 1/n_s and
 * the mean term.  A sample whose occupation is not a configuration of the
 * sector (not strictly ascending, an up orbital >= n_sites, a down orbital
 * outside n_sites .. M-1) is skipped: its t_s is NaN and it adds nothing to
 * out; the call still returns VMC_OK.  Sizes beyond the scratch (n_sites > 64) and bad strides or
 * pointers return INVALID_ARG (vmc_last_error_detail says which).  The first
 * call on each device looks up the scratch's device address with that device
 * current (cudaGetSymbolAddress), so make that first call before any stream
 * capture.  Every call shares the one scratch array: calls that overlap on the
 * GPU (other streams, other threads) race and must be serialised by the
 * caller; a call overwrites all of the scratch it reads, so nothing needs
 * clearing between calls. */
int sr_pairing_product_noalloc(int64_t n_s, int n_sites, int n_up, int n_dn, const uint8_t* occ,
                               int64_t occ_stride, const float* pf, int64_t pf_stride, const float* v, float* t,
                               double* out, void* stream);

/* Product paths of the BF16-store S product (no counterpart in the paper:
 * the same Eq. 7 arithmetic organised in different passes).
 *   VMC_PATH_SORTED  two passes over index-carrying copies built once per set
 *                    of samples: a sample-major gather of t_s = O_s . v, then
 *                    a parameter-major sum of t_s O_s (no atomics);
 *   VMC_PATH_FUSED   one vector only: one pass over the sample-major copy,
 *                    scattering t_s O_s into private shared-memory images;
 *   VMC_PATH_STAGED  one or two vectors: a per-sample pass over the store
 *                    itself, samples staged in shared memory by bulk copies;
 *   VMC_PATH_GENERIC the plain per-sample pass (any number of vectors);
 *   VMC_PATH_COMPACT one vector only: the two-pass product whose gather reads
 *                    a copy of the 2-byte values alone (in the row-major
 *                    order of electron pairs) and forms each element's index
 *                    from the sample's occupation; more than one vector takes
 *                    VMC_PATH_SORTED.
 * A path that does not apply to a problem falls back to the next applicable
 * one in the order SORTED, FUSED, STAGED, GENERIC (COMPACT to SORTED).
 * VMC_PATH_STAGED / GENERIC also select the pass of the FP32 store with FP32
 * accumulation. */
#define VMC_PATH_AUTO 0
#define VMC_PATH_SORTED 1
#define VMC_PATH_FUSED 2
#define VMC_PATH_STAGED 3
#define VMC_PATH_GENERIC 4
#define VMC_PATH_COMPACT 5
int vmc_set_product_path(vmc_handle h, int path);

typedef struct {
    int path;        /* fastest one-vector path (VMC_PATH_*), used under AUTO     */
    int path4;       /* fastest four-vector path, used under AUTO for 2 and 4     */
    double ms[6];    /* mean time of one one-vector product per path, < 0 if n/a  */
    double ms4[6];   /* the same for four vectors                                 */
} vmc_tune_info;

/* Autotuner: times `reps` BF16 products of one and of four vectors on every
 * applicable path over the handle's current samples (CUDA events on
 * `stream`, after one warm-up product that also builds the path's copies)
 * and makes the fastest the handle's AUTO choice.  info (host, may be NULL)
 * receives the timings.  Errors: STATE (no samples or no BF16 store). */
int sr_autotune(vmc_handle h, int reps, vmc_tune_info* info, void* stream);
/* Set the AUTO choice directly (a choice sr_autotune made earlier for the
 * same workload, e.g. read back from a cache): one-vector products on
 * `path`, two- and four-vector products on `path4` (VMC_PATH_SORTED ..
 * VMC_PATH_COMPACT). */
int vmc_set_auto_paths(vmc_handle h, int path, int path4);

/* Failure detection (no counterpart in the paper).  The streaming products
 * stage samples in shared memory with bulk copies and wait for each copy a
 * bounded number of times (mbarrier try-wait); a wait that runs out makes
 * the kernel drain its own copies and stop, and the call returns
 * VMC_ERR_TIMEOUT instead of hanging (sr_apply_S reads the kernels' status
 * word before it returns; sr_cg_solve at its next convergence check).  This
 * sets the number of tries of those waits (default 4,194,304); the drain
 * before a kernel exits always uses the default.  A caller that must bound
 * the time a product can wait on memory lowers it; 0 makes every wait give
 * up at once (every staged product then returns VMC_ERR_TIMEOUT). */
int vmc_set_wait_limit(vmc_handle h, uint32_t tries);

const char* vmc_error_string(int code);
/* Text of the last failing CUDA call or internal check on the calling
 * thread, for diagnostics ("" if none).  The pointer stays valid until the
 * next failing call on that thread. */
const char* vmc_last_error_detail(void);

#ifdef __cplusplus
}
#endif
#endif
