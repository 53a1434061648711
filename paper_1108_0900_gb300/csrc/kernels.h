// Kernel argument blocks and launch wrappers shared by the vmcsr translation
// units.  Internal to the library; the public boundary is include/vmcsr.h.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace vmc {

// Walker kernel (sampling, measurement of given configurations, adjoint).
struct SampleArgs {
    DevProblem pb;
    int n_walkers;        // warps launched (walkers or given configurations)
    int spw;              // measurements per walker
    int n_burn;           // sweeps before the first measurement
    int props_per_sweep;  // N for sampling, 0 to only measure
    int write_back;       // 1: write the final configuration / counter back
    int refresh_every;    // sweeps between from-scratch rebuilds of the inverse (0: call start only)
    int want_energy;
    uint64_t seed;
    uint8_t* walker_occ;  // [n_walkers][N] ascending on entry
    uint64_t* walker_step;
    int XS;               // row stride of the inverse in shared memory
    int GS;               // row stride of G (ab initio local energy)
    int ncorr_pad;
    size_t warp_bytes;
    // O store
    uint8_t* s_occ;       // [n_s][Nst]
    int Nst;
    cstate_t* s_cidx;     // [n_s][ncst]
    int ncst;
    double* s_E;
    double* s_lnrun;      // [n_s] the chain's running ln|Psi| since the call started (may be null)
    double* s_pf64;
    float* s_pf32;
    __nv_bfloat16* s_pf16;
    int64_t Pst;
    // adjoint mode: bgrad[k] += bw[s] O_k(n_s) instead of writing the store
    const double* bw;
    double* bgrad;
    int* status;
};

struct LogPsiArgs {
    DevProblem pb;
    int64_t n_s;
    const uint8_t* s_occ;
    int Nst;
    const cstate_t* s_cidx;
    int ncst;
    int XS;
    size_t warp_bytes;
    double* out;
};

template <typename R> __global__ void k_walkers(SampleArgs a);
cudaError_t launch_walkers_batch(bool fp64, int blocks, int threads, size_t smem, cudaStream_t st,
                                 const SampleArgs* args, const int* wstart, int n, size_t warp_bytes);
__global__ void k_logpsi(LogPsiArgs a);

// ---------------------------------------------------------------------------
// SR kernels
// ---------------------------------------------------------------------------
enum StoreKind { STORE_F64 = 0, STORE_F32 = 1, STORE_BF16 = 2 };

// Streaming pass over the O store.  With GATHER, t_s = O_s . V for K vectors
// (correlator gather + pairing-block dot) is computed and written to T;
// otherwise t_s is read from T.  Then sum_s t_s O_s restricted to the
// pairing block is accumulated per CTA and written to pf_partial[cta].
template <typename AT>
struct MainArgs {
    DevProblem pb;
    int64_t n_s;
    const uint8_t* s_occ;
    int Nst;
    const cstate_t* s_cidx;
    int ncst;
    const void* s_pf;
    int64_t Pst;
    const AT* V;          // [K][nv]
    const AT* invC;       // [ncp]
    AT* T;                // [n_s][K]
    AT* pf_partial;       // [gridDim][npf][K]
    const int* stop;      // early exit flag (may be null)
};

template <typename AT>
struct CorrArgs {
    DevProblem pb;
    int64_t n_s;
    const cstate_t* cidxT;  // [ncorr][n_s]
    const AT* T;            // [n_s][K]
    AT* corr_raw;           // [ncp][K] sum over samples of t_s per state (zeroed by the caller)
    const int4* units;      // cluster work units (class, first, end into class_inst)
    const int* stop;
};

constexpr int kCorrCluster = 8;  // CTAs per correlator (one thread-block cluster)

template <typename AT, typename VT>
struct FinArgs {
    DevProblem pb;
    int64_t n_s;
    double inv_n;           // 1 / n_s
    int centered;           // the pass scattered t_s - Obar . V: skip the Obar term
    const AT* pf_partial;
    const AT* pf_raw;       // [npf][K] pairing-block sums
    const AT* corr_raw;     // [ncp][K] correlator sums
    const AT* ObarA;        // [nv] Obar in AT (S mode, uncentered)
    const AT* invC;
    const double* obv_part; // [nblk][K] partial dots Obar . V (S mode, uncentered)
    int n_obv_part;
    const VT* V;            // [K][nv]
    double shift;
    VT* out;                // [K][nv]
    double* dot_part;       // [gridDim][K] partial out . V (may be null)
    // gradient mode
    double* Obar_out;
    double* g_out;
    const double* E_sum;    // [nblk] partial sums of E (gradient mode)
    int n_E_part;
    const int* stop;
};


template <typename ST, typename AT, int K, bool GATHER>
__global__ void __launch_bounds__(512) k_sr_main(MainArgs<AT> a);
cudaError_t launch_sr_main_batch(int store_bytes, int blocks, size_t smem, cudaStream_t st,
                                 const MainArgs<double>* args, const int* cta0, int n);
template <typename AT, int K>
__global__ void __cluster_dims__(kCorrCluster, 1, 1) __launch_bounds__(256) k_corr_scatter(CorrArgs<AT> a);
template <typename AT, int K> __global__ void __launch_bounds__(256) k_corr_scatter_global(CorrArgs<AT> a);
template <typename AT, typename VT, int K> __global__ void __launch_bounds__(256) k_finalize_S(FinArgs<AT, VT> a);
template <typename AT> __global__ void __launch_bounds__(256) k_finalize_grad(FinArgs<AT, double> a);
__global__ void k_build_T_grad(const double* E, int64_t n_s, double* T, double* E_part);
template <typename TA, typename TB, int K>
__global__ void __launch_bounds__(256) k_dot_part(const TA* x, const TB* y, int64_t n, double* part, const int* stop);
template <typename AT>
__global__ void __launch_bounds__(256) k_reduce_pf(const AT* part, int nblk, int npfK, AT* raw);
__global__ void k_transpose_cidx(const cstate_t* cidx, int ncst, int ncorr, int64_t n_s, cstate_t* cidxT);
template <typename VT> __global__ void k_cast(const double* src, VT* dst, int64_t n, double scale);

// conjugate-gradient scalars (FP64, device): rr, |b|^2, tol^2 |b|^2,
// iterations, rr of the previous step
// fused CG update after a centered product (see k_cg_fxr)
template <typename VT>
struct CgFusedArgs {
    VT* x;
    VT* r;
    const VT* p;
    const VT* pf_raw;       // [npf] pairing sums of the centered pass
    VT* corr_raw;           // [ncp] correlator sums (zeroed after reading)
    const VT* invC;         // [ncp]
    int64_t n, ncp;
    double inv_n, shift;
    const double* tt_part;  // partial sums of centered t_s^2 (gather)
    int ntt;
    const double* pp_part;  // partial sums of |p|^2
    int npp;
    double* scal;
    double* rr_part;        // out: partial r . r
    const int* stop;
};

// SR parameter update (k_sr_update)
struct UpdateArgs {
    double* C64;
    float* C32;
    double* invC64;
    float* invC32;
    double* F64;            // [M][M] antisymmetric
    float* F32;
    const uint32_t* pq_of;  // [npf] p | q << 16 of pairing index rowbase(p) + q
    const double* y;        // [nv] solution of (S + eps) y = g
    int64_t ncp, npf;
    int M;
    double tau, inv_n;
    const double* e_part;   // partial sums of E_L
    int ne;
    const double* oy_part;  // partial sums of Obar . y
    int noy;
    double* x0;             // out: x_0
    int* status;
};

enum { CG_RR = 0, CG_BB = 1, CG_TOL2 = 2, CG_IT = 3, CG_RRP = 4 };
template <typename VT>
__global__ void __launch_bounds__(256) k_cg_init(const VT* b, VT* x, VT* r, VT* p, int64_t n, double* part);
__global__ void k_cg_start(const double* part, int npart, double* scal, double tol, int* stop);
template <typename VT>
__global__ void __launch_bounds__(256) k_cg_xr(VT* x, VT* r, const VT* p, const VT* Ap, int64_t n,
                                               const double* pAp_part, int npart, double* scal,
                                               double* rr_part, int* stop);
template <typename VT>
__global__ void __launch_bounds__(256) k_cg_p(const VT* r, VT* p, int64_t n, const double* rr_part, int npart,
                                              double* scal, const VT* Obar, double* obp_part, double* pp_part,
                                              int* stop, int max_iter);
template <typename VT> __global__ void __launch_bounds__(256) k_cg_fxr(CgFusedArgs<VT> a);
template <typename VT>
__global__ void __launch_bounds__(256) k_cg_fxrp(CgFusedArgs<VT> a, const VT* Obar, double* obp_part, int* stop,
                                                 int max_iter);
template <typename VT>
__global__ void __launch_bounds__(256) k_cg_fxrp1(CgFusedArgs<VT> a, const VT* Obar, double* obp_part, int* stop,
                                                 int max_iter);
__global__ void k_sub(const double* a, const double* b, double* y, int64_t n, double* part);
__global__ void __launch_bounds__(256) k_vec_sum(const double* x, int64_t n, double* part);
__global__ void __launch_bounds__(256) k_uncenter(double* out, const double* Obar, const double* obv_part, int nobv,
                                                  double n_s, int64_t nv);
__global__ void __launch_bounds__(256) k_sr_update(UpdateArgs a);
__global__ void k_axpby(double a, const double* x, double b, double* y, int64_t n);
template <typename VT> __global__ void k_axpy_to64(double* x, const VT* d, double scale, int64_t n);

}  // namespace vmc

namespace vmc {

// TMA-staged streaming pass (FP32 accumulation, BF16 or FP32 store): every
// warp double-buffers its samples' O records in shared memory with 1-D bulk
// copies and walks the pairing block row by row.
struct StreamArgs {
    DevProblem pb;
    int64_t n_s;
    const uint8_t* s_occ;
    int Nst;
    const cstate_t* s_cidx;
    int ncst;
    const void* s_pf;
    int64_t Pst;
    int st_bytes;           // element size of the store
    const float* V;         // [K][nv]
    const float* invC;
    float* T;               // [n_s][K]
    float* pf_partial;      // [gridDim][npf][K]
    const int* stop;
    int* status;            // ST_TIMEOUT on a wait that ran out
    uint32_t spin_limit;    // tries of each bounded wait on a staged sample
    size_t buf_bytes;       // one staging buffer (occ | pf)
};

template <typename ST, int K> __global__ void __launch_bounds__(768, 1) k_sr_stream(StreamArgs a);
__global__ void __launch_bounds__(512, 1) k_sr_stream_bf16c(StreamArgs a);

}  // namespace vmc

namespace vmc {

// Sorted two-pass product over the BF16 store (sorted.cu).
struct SortedArgs {
    DevProblem pb;
    int64_t n_s;
    const cstate_t* s_cidx;
    int ncst;
    const uint32_t* G;      // [n_s][Pst] (pq << 16) | bf16
    int64_t Pst;
    const float* V;         // [K][nv]
    const float* invC;
    const double* obv_part; // [n_obv_part][K] partial dots Obar . V (centering)
    int n_obv_part;
    float* Tv;              // [n_s][K] centered per-sample dots O_s . V - Obar . V
    const uint32_t* T;      // parameter-major (s_local << 16) | bf16, per chunk of kTChunk samples
    const uint32_t* base;   // [nchunk][npf + 1] run offsets
    int nchunk;
    int pq_per_cta;         // pairing parameters of one scatter CTA (in one chunk)
    int corr_in_cta;        // the pairing CTAs build the correlator histograms of their chunk
    int hist_cap;           // floats of the in-CTA histogram region
    int hist_off;           // its byte offset in the scatter's dynamic shared memory
    float* part;            // [nchunk][npf][K] per-chunk pairing sums (nchunk > 1)
    unsigned* done;         // [parameter groups] chunks finished so far (0 between launches)
    float* raw;             // [npf][K] scatter result
    const uint32_t* Tc;     // correlator runs: sample << 5 | k mod 32, grouped by parameter k
    const uint32_t* cbase;  // [ncp + 1] run offsets
    const uint2* items;     // correlator work items (group, first entry)
    const uint32_t* n_items;// device count of items
    int ncb;                // CTAs of the correlator part (8 items each)
    float* craw;            // [ncp][K] correlator sums (without the 1/C factor), zeroed by the caller
    double* tt_part;        // [gridDim] partial sums of centered t_s^2 (K = 1; may be null)
    const int* stop;
    // correlator half as shared-memory histograms: CTAs [0, nhist) take
    // (class, sample slice) = (b / hist_slices, b % hist_slices); when nhist is
    // 0 the ncb CTAs of correlator work items do it instead
    int nhist;
    int hist_slices;
    const cstate_t* cidxT;  // [ncorr][n_s] correlator states, correlator-major
};

constexpr int kCorrPerLane = 4;    // the sorted gather handles up to 128 correlators
constexpr int kTRun = 128;         // T runs are padded to whole blocks of this many entries
constexpr int kTChunk = 8192;      // samples per T chunk: the scatter stages a chunk's t_s in shared memory
constexpr int kScatterMaxPQ = 4096; // parameters of one scatter CTA at most (their run ends sit in shared memory)
constexpr int kCorrItem = 2048;    // entries per correlator work item of the sorted scatter
constexpr int kInstPerUnit = 4;    // correlators of one class per cluster of the histogram scatter

constexpr int kGParts = 4;         // parts of consecutive pq per G row (warps per image of the single pass)
__global__ void __launch_bounds__(256) k_build_G(DevProblem pb, int64_t n_s, const uint8_t* s_occ, int Nst,
                                                 const __nv_bfloat16* pf16, int64_t Pst, const uint32_t* fulltab,
                                                 int wq, int64_t Gst, uint32_t* G, uint16_t* G16, int64_t Gst16);
constexpr int kCompactThreads = 512;   // threads per CTA of the compact gather
template <int U>
__global__ void __launch_bounds__(512) k_gather_C(SortedArgs a, const uint16_t* G16, int64_t Gst16,
                                                 const uint16_t* wtab, const uint8_t* s_occ, int Nst);
__global__ void __launch_bounds__(512) k_count_G(const uint32_t* G, int64_t Pst, int P, int64_t s_begin,
                                                 int64_t s_end, int npf, uint32_t* counts);
__global__ void k_scan_blocks(uint32_t* counts, int nblk, int npf, uint32_t* total);
__global__ void __launch_bounds__(1024) k_scan_params(const uint32_t* total, int npf, uint32_t base0, uint32_t* base);
__global__ void __launch_bounds__(256) k_rank_T(uint32_t* T, int64_t t_chunk, int nchunk, const uint32_t* base,
                                                int npf, int64_t n_s);
__global__ void __launch_bounds__(512) k_fill_T(const uint32_t* G, int64_t Pst, int P, int64_t s_begin,
                                                int64_t s_end, int npf, const uint32_t* offs, const uint32_t* base,
                                                uint32_t* T);
// threads per CTA of the sorted gather: one v table per CTA, so the
// one-vector gather runs few, large CTAs, which leaves L1 to the G stream
// (512 threads with the next row prefetched measured best)
constexpr int gather_threads(int K) { return K == 1 ? 512 : 256; }
template <int K, int U> __global__ void __launch_bounds__(gather_threads(K)) k_gather_G(SortedArgs a);
// threads per CTA of the sorted scatter: the four-vector chunk table (128 KB)
// leaves room for one CTA per SM, which then runs 16 warps
constexpr int scatter_threads(int K) { return K == 4 ? 512 : 256; }
// the one-vector chunk table (32 KB) leaves room for six CTAs per SM
constexpr int scatter_min_ctas(int K) { return K == 1 ? 6 : 1; }
template <int K>
__global__ void __launch_bounds__(scatter_threads(K), scatter_min_ctas(K)) k_scatter_T(SortedArgs a);
__global__ void __launch_bounds__(512) k_count_C(DevProblem pb, int64_t n_s, const cstate_t* cidxT,
                                                 uint32_t* ccount, int shared_hist);
__global__ void __launch_bounds__(512) k_fill_C(DevProblem pb, int64_t n_s, const cstate_t* cidxT,
                                                uint32_t* cursor, uint32_t* Tc);
__global__ void k_corr_item_count(const uint32_t* cbase, int64_t ncp, uint32_t* n_items);
__global__ void k_corr_item_fill(const uint32_t* cbase, int64_t ncp, const uint32_t* item_base, uint2* items);

// Fused single-pass product over the sorted BF16 rows G, one vector
// (fused.cu): per sample the gather t_s = O_s . v and, in the same pass, the
// scatter of t_s O_s into a private shared-memory image of the pairing block
// per warp (no atomics, no parameter-major copy).
constexpr int kFusedImages = 6;   // private pairing images per CTA (one per group of kGParts warps)
constexpr int kFusedWarps = kFusedImages * kGParts;
constexpr int kFusedAhead = 4;    // rows per group requested into L2 ahead of the register loads
template <int U> __global__ void __launch_bounds__(kFusedWarps * 32, 1) k_sv_fused(SortedArgs a, float* pf_partial,
                                                                                 int wq);
__global__ void __launch_bounds__(256) k_sv_finish(SortedArgs a, const float* pf_partial, int nblk);

// ---------------------------------------------------------------------------
// accelerated linear method (Sec. II.B): Eq. 10 products with the basis
// {Psi, Psi^1 .. Psi^nv} from a stored sample set (lm.cu)
// ---------------------------------------------------------------------------
struct LmArgs {
    DevProblem pb;
    int64_t n_s;
    const uint8_t* s_occ;   // [n_s][Nst] ascending occupied spin orbitals
    int Nst;
    const cstate_t* s_cidx; // [n_s][ncst]
    int ncst;
    const void* pf;         // [n_s][Pst] pairing block in the kernel's precision R
    int64_t Pst;
    const double* x;        // [nv + 1]: x_0 then the parameter block
    const void* Xt;         // [M][M] antisymmetric matrix of the pairing part of x (R)
    const void* xc;         // [ncp] x_k / C_k for the correlator part of x (R)
    int n_mu;               // factor pairs of Eq. 9, each a sparse ns x ns matrix:
    const int* Lptr;        // [n_mu + 1] rows of the nonzeros of L^mu
    const int* Lidx;        // i ns + j of each nonzero
    const void* Lval;       // its value (R)
    const int* Rptr;        // the same for R^mu
    const int* Ridx;
    const void* Rval;
    double c0;
    double inv_n;
    double* Hx;             // [nv + 1], accumulated (zeroed by the caller)
    double* Sx;             // [nv + 1] or null
    int XS, GS;             // row strides of the per-warp matrices
    int warp_bytes;
};
size_t lm_warp_bytes(int N, int M, int ns, int n_mu, int ncorr, int elem);
template <typename R> __global__ void k_lm_prep(DevProblem pb, const double* x, R* Xt, R* xc);
template <typename R> __global__ void k_lm_apply(LmArgs a);
template <typename R> __global__ void k_lm_diag(LmArgs a, double* d);
__global__ void k_lm_dots(const double* V, int64_t ld, int k, const double* u, int64_t n, double* part);
__global__ void k_lm_dots_reduce(const double* part, int nb, int k, double* out);
__global__ void k_lm_combine(double* out, const double* V, int64_t ld, int k, const double* c, int64_t n, double alpha);
__global__ void k_lm_precond(double* t, const double* r, const double* d, double eps, int64_t n);
__global__ void k_lm_update(UpdateArgs a, const double* x, double scale);

// enlarged block CG (bcg.cu): [4][n] FP32 block vectors, FP64 4 x 4 algebra
__global__ void k_bcg_split(const float* b, float* B, int64_t n, int64_t ncp, int64_t corr_split,
                            const uint32_t* pq_of, int ns);
// device state of the block CG iteration (bcg.cu)
struct BcgState {
    double RR[16];     // R^T R of the current residual block
    double al[16];     // alpha = (P^T Q)^{-1} R^T R
    double be[16];     // beta = (R^T R)^{-1} R_new^T R_new
    double b2, thr;    // |b|^2 of the column sum, and the stopping threshold itol^2 b2
    int it, steps;     // products, completed steps
    int breakdown;     // a singular 4 x 4 step system stopped the solve
};
__global__ void k_bcg_gram(const float* U, const float* V, int64_t n, double* part, const int* stop);
__global__ void k_bcg_start(const double* part, int nb, BcgState* S, double itol);
__global__ void k_bcg_alpha(const double* part, int nb, BcgState* S, int* stop);
__global__ void k_bcg_beta(const double* part, int nb, BcgState* S, int* stop, int max_iter);
__global__ void k_bcg_step(float* X, float* R, const float* P, const float* Q, const BcgState* S, int64_t n,
                           double* part, const int* stop);
__global__ void k_bcg_dir(float* P, const float* R, const BcgState* S, const double* Obar, int64_t n,
                          double* obv_part, const int* stop);

}  // namespace vmc
