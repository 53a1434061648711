// Host side of the vmcsr C ABI (include/vmcsr.h): handle lifetime, problem
// tables, kernel launches and the conjugate-gradient drivers.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.h"
#include "vmcsr.h"

using namespace vmc;

namespace {

constexpr int kMaxK = 4;
constexpr int kNumPart = 256;   // blocks of the reduction kernels
constexpr int kChunk = 16;      // CG iterations between host convergence checks
constexpr int kBlockInnerMax = 4096;   // block CG steps of one inner solve at most
constexpr int kScalX0 = 7;      // d_scal slot of the SR update's x_0
constexpr int kMaxBatch = 16;   // problems per batched launch

#define VCK(x)                                                    \
    do {                                                          \
        cudaError_t e_ = (x);                                     \
        if (e_ != cudaSuccess) {                                  \
            set_err(std::string(#x) + ": " + cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? VMC_ERR_OOM : VMC_ERR_CUDA; \
        }                                                         \
    } while (0)

thread_local std::string g_err;
void set_err(const std::string& s) { g_err = s; }

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace

struct vmc_ctx {
    int dev = 0, nsm = 0;
    size_t smem_optin = 0;
    int ns = 0, M = 0, nu = 0, nd = 0, N = 0, ncorr = 0, P = 0, npf = 0;
    int64_t ncp = 0, nv = 0;
    int n_walkers = 0, spw = 0;
    int64_t ncap = 0, n_s = 0;
    int wprec = VMC_FP64, keep64 = 1, keeplow = 0, refresh_every = 0, fp64_refresh = 0;
    int ham = 0;
    int maxd = 1;
    int max_csites = 0;          // sites of the largest correlator
    bool ff_sums = true;         // FP32-store passes with FP64 sums in FP32-pair arithmetic
    // shared-memory carveout of the FP32 ab initio walkers in percent: 58 (two
    // 4-walker CTAs per SM, more L1 for the tables) measured 213 ms against
    // 221 ms at the driver's choice and 333 ms at 30 (24 orbitals, 65,536 samples)
    int walker_carveout_ab = 58;
    bool params_set = false, walkers_set = false;
    bool use_stream = true;     // TMA-staged pass for FP32-accumulation products
    bool stream_cached = false;  // register-cached variant for BF16, one vector (slower: 16 warps)
    bool use_sorted = true;      // sorted two-pass product for the BF16 store
    int last_gather_grid = 0;    // CTAs (tt partials) of the last sorted gather
    bool sorted_ok = false;      // G / T built for the current samples
    bool use_fused = true;       // fused single-pass product over G (BF16 store, one vector)
    bool use_compact = true;     // two-pass product with the compact gather over G16 (one vector)
    bool use_coop_update = true; // inner CG: x/r and p updates as one cooperative launch
    bool rank_T = true;          // bank order inside T's blocks (k_rank_T)
    struct SortedLaunch {        // launch shapes of the sorted product for one K (see plan_sorted)
        int64_t n_s = -1;
        bool compact = false;
        int ggrid = 0, sgrid = 0;
        size_t gsmem = 0, ssm = 0;
        int nhist = 0, hist_slices = 1, ncb = 0, corr_in_cta = 0, hist_cap = 0, hist_off = 0, pq_per_cta = 1;
    } sorted_launch[3];
    bool coop_launch = false;    // the device supports cooperative launches
    int path = VMC_PATH_AUTO;    // product path set by the caller (VMC_PATH_*)
    int auto_path = VMC_PATH_SORTED;   // one-vector BF16 path used under AUTO (sr_autotune may change it)
    int auto_path4 = VMC_PATH_SORTED;  // two- and four-vector BF16 path used under AUTO
    bool g_ok = false;           // G built for the current samples
    bool corr_ok = false;        // correlator runs built for the current samples
    uint32_t wait_limit = 1u << 22;  // tries of each bounded wait on a staged sample
    double itol_floor = 0.0;     // inner relative tolerance floor of the mixed solves (0: default)
    int last_fused_grid = 0;     // CTAs (tt partials) of the last fused pass
    int sort_nblk = 0, sort_nchunk = 0;
    size_t t_chunk = 0;          // T entries reserved per chunk of kTChunk samples
    bool obar_ok[3] = {false, false, false};  // per store: FP64, FP32, BF16
    std::vector<int64_t> corr_off;

    DevProblem pb{};
    // device tables
    int *d_corr_ptr = nullptr, *d_corr_sites = nullptr;
    int64_t* d_corr_off = nullptr;        // [ncorr + 1] first parameter of each correlator's block, then ncp
    int64_t* d_class_off = nullptr;       // [n_class + 1] parameter blocks of the classes
    int* d_class_ptr = nullptr;           // [n_class + 1] into d_class_inst
    int* d_class_inst = nullptr;          // correlators grouped by class
    int n_class = 0;
    int4* d_units = nullptr;              // histogram-scatter work units (class, first, end)
    int n_units = 0;
    uint2* d_items = nullptr;             // sorted correlator-scatter work items (group, first entry)
    uint32_t* d_nitems = nullptr;         // items per group
    uint32_t* d_item_base = nullptr;      // [groups + 1] exclusive scan, total at the end
    int64_t max_items = 0;
    int *d_site_cptr = nullptr, *d_site_corr = nullptr, *d_site_w = nullptr;
    uint32_t* d_corr_site_w = nullptr;
    uint32_t* d_pq_of = nullptr;   // pairing index -> p | q << 16
    int *d_nbr_ptr = nullptr, *d_nbr_site = nullptr;
    double* d_nbr_t = nullptr;
    double *d_h64 = nullptr, *d_eri64 = nullptr;
    float *d_h32 = nullptr, *d_eri32 = nullptr;
    int *d_pair_ptr = nullptr, *d_pair_corr = nullptr;
    uint16_t* d_dexc = nullptr;   // double-excitation pair tables (ab initio)
    bool pair_unique = false;     // no site pair lies in two correlators (and ncp < 2^30)
    double *d_C64 = nullptr, *d_invC64 = nullptr, *d_F64 = nullptr;
    float *d_C32 = nullptr, *d_invC32 = nullptr, *d_F32 = nullptr;
    uint16_t* d_pairtab = nullptr;
    uint32_t* d_fulltab = nullptr;   // [P] full row-major rank -> block index e | a << 16 | b << 24
    int64_t Gst = 0;                 // row stride of G (kGParts regions of gwq 16-byte words)
    int gwq = 0;
    int* d_rowbase = nullptr;
    // walkers
    uint8_t* d_wocc = nullptr;
    uint64_t* d_wstep = nullptr;
    uint8_t* d_mocc = nullptr;  // configurations handed to measure / backward
    // O store
    int Nst = 0, ncst = 0;
    int64_t Pst = 0;
    uint8_t* d_socc = nullptr;
    cstate_t *d_cidx = nullptr, *d_cidxT = nullptr;
    double* d_E = nullptr;
    double* d_lnrun = nullptr;   // [ncap] chains' running ln|Psi| at each stored sample
    double* d_Echain = nullptr;  // [ncap] E_L of the FP32 chains before an FP64 refresh
    bool refreshed = false;      // the stored samples come from an FP64 refresh
    double* d_lnps = nullptr;    // [ncap] scratch for vmc_sample_stats
    unsigned char* d_batch = nullptr;   // argument blocks of batched launches led by this handle
    size_t batch_bytes = 0;
    double* d_pf64 = nullptr;
    float* d_pf32 = nullptr;
    __nv_bfloat16* d_pf16 = nullptr;
    double* d_Obar[3] = {nullptr, nullptr, nullptr};
    float* d_Obar32[3] = {nullptr, nullptr, nullptr};   // FP32 copies for the inner solve
    int* d_status = nullptr;
    // scratch
    void* d_T = nullptr;
    void* d_pfpart = nullptr;
    size_t pfpart_bytes = 0;
    double* d_corrraw = nullptr;   // [ncp][kMaxK] correlator sums of a pass (FP64 or FP32)
    double* d_part = nullptr;   // 8 slots x kNumPart x kMaxK
    double* d_pfraw = nullptr;  // [npf][K] reduced pairing-block sums (FP64 or FP32 per pass)
    uint32_t *d_G = nullptr, *d_Tsort = nullptr, *d_counts = nullptr, *d_total = nullptr, *d_base = nullptr;
    uint16_t* d_G16 = nullptr;   // [ncap][Gst16] BF16 values in the row-major pair order (compact gather)
    uint16_t* d_wtab = nullptr;  // [Gst16 / 8] pair (a | b << 8) of the first value of each 16-byte word
    int64_t Gst16 = 0;
    float* d_tpart = nullptr;    // [chunks][npf][kMaxK] per-chunk pairing sums of the sorted scatter
    bool scatter_corr_front = true;   // correlator items of the sorted scatter as CTAs of their own
    bool scatter_corr_hist = true;    // correlator half of the sorted scatter as class histograms
    int scatter_in_cta_mink = 2;      // vectors from which the pairing CTAs build the correlator histograms
    // waves of pairing CTAs of the sorted scatter: one wave left a tail behind
    // the histogram CTAs inside the SR step (one vector, 8x8 / 2x3: 137.7 ms per
    // step at one wave, 131.1 at two, 128.2 at three); four vectors (one CTA
    // per SM) measured best at one wave (0.394 against 0.415 ms at three)
    int scatter_waves1 = 3, scatter_waves4 = 1;
    unsigned* d_tdone = nullptr; // [npf] chunks finished per parameter group (0 between launches)
    uint32_t *d_Tc = nullptr, *d_ccount = nullptr, *d_cbase = nullptr;   // correlator runs
    double* d_scal = nullptr;
    int* d_stop = nullptr;
    // CG vectors
    double *d_x64 = nullptr, *d_r64 = nullptr, *d_p64 = nullptr, *d_q64 = nullptr, *d_t64 = nullptr;
    float *d_x32 = nullptr, *d_r32 = nullptr, *d_p32 = nullptr, *d_q32 = nullptr, *d_b32 = nullptr;
    double* h_pinned = nullptr;  // small host staging
    // linear method: the Hamiltonian as c0 + sum_mu Lhat_mu Rhat_mu (Eq. 9),
    // spatial factors [n_mu][ns][ns] built at creation, uploaded on first use
    int lm_nmu = 0;
    double lm_c0 = 0.0;
    std::vector<double> lm_L, lm_R;
    double *d_lmL64 = nullptr, *d_lmR64 = nullptr, *d_lmXt = nullptr, *d_lmxc = nullptr;
    float *d_lmL32 = nullptr, *d_lmR32 = nullptr;
    int *d_lmLptr = nullptr, *d_lmLidx = nullptr, *d_lmRptr = nullptr, *d_lmRidx = nullptr;
    // Davidson workspace: basis V and its images (column-major, ld = lm_ld),
    // work vectors, dot partials
    double* d_bcg = nullptr;   // block CG: Gram partials, reduced Gram, alpha, beta
    int lm_cap = 0;
    int64_t lm_ld = 0;
    double *d_lmV = nullptr, *d_lmHV = nullptr, *d_lmSV = nullptr, *d_lmW = nullptr, *d_lmdot = nullptr;

    // measurement support (vmc_profile)
    bool prof = false;
    int64_t n_launch = 0;
    struct PassRec { cudaEvent_t a, b; int kind; double bytes; };
    std::vector<PassRec> recs;
    std::vector<cudaEvent_t> ev_pool;
    double acc_ms[4] = {0, 0, 0, 0}, acc_bytes[4] = {0, 0, 0, 0};
    int64_t acc_n[4] = {0, 0, 0, 0};
    cudaEvent_t get_event() {
        if (!ev_pool.empty()) { cudaEvent_t e = ev_pool.back(); ev_pool.pop_back(); return e; }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }

    std::vector<void*> allocs;
    template <typename T> cudaError_t alloc(T** p, size_t count) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) { allocs.push_back(q); *p = (T*)q; }
        return e;
    }
    double* part(int slot) { return d_part + (size_t)slot * kNumPart * kMaxK; }
};

extern "C" const char* vmc_error_string(int code) {
    switch (code) {
        case VMC_OK: return "ok";
        case VMC_ERR_INVALID_ARG: return "invalid argument";
        case VMC_ERR_OOM: return "out of device memory";
        case VMC_ERR_SINGULAR: return "singular pairing submatrix or zero correlator amplitude";
        case VMC_ERR_NONFINITE: return "non-finite value";
        case VMC_ERR_NOT_CONVERGED: return "solver did not reach the tolerance";
        case VMC_ERR_TIMEOUT: return "timeout";
        case VMC_ERR_CUDA: return "CUDA error";
        case VMC_ERR_UNSUPPORTED: return "unsupported configuration";
        case VMC_ERR_STATE: return "call out of order (parameters, walkers or samples missing)";
        default: return "unknown error";
    }
}

extern "C" const char* vmc_last_error_detail(void) { return g_err.c_str(); }

namespace vmc {
void set_error_detail(const std::string& s) { set_err(s); }
}  // namespace vmc

// ---------------------------------------------------------------------------
// creation
// ---------------------------------------------------------------------------
extern "C" int vmc_create(const vmc_lattice* lat, const vmc_hamiltonian* ham, const vmc_ansatz* ans,
                          const vmc_options* opt, vmc_handle* out) {
    if (!lat || !ham || !ans || !opt || !out) return VMC_ERR_INVALID_ARG;
    *out = nullptr;
    const int ns = lat->n_sites, nu = ans->n_up, nd = ans->n_dn, N = nu + nd;
    if (ns < 1 || ns > 64 || nu < 0 || nd < 0 || nu > ns || nd > ns || N < 2 || (N & 1) || N > 64)
        return VMC_ERR_INVALID_ARG;
    if (opt->n_walkers < 1 || opt->samples_per_walker < 1) return VMC_ERR_INVALID_ARG;
    if (opt->walker_precision != VMC_FP64 && opt->walker_precision != VMC_FP32) return VMC_ERR_INVALID_ARG;
    if (ham->kind != VMC_HUBBARD && ham->kind != VMC_ABINITIO) return VMC_ERR_INVALID_ARG;
    if (ham->kind == VMC_ABINITIO && (!ham->h || !ham->chol || ham->n_chol < 1)) return VMC_ERR_INVALID_ARG;
    if (ans->n_corr < 0 || (ans->n_corr > 0 && (!ans->corr_ptr || !ans->corr_sites))) return VMC_ERR_INVALID_ARG;
    if (lat->n_bonds < 0 || (lat->n_bonds > 0 && (!lat->bonds || !lat->bond_t))) return VMC_ERR_INVALID_ARG;

    vmc_ctx* h = new vmc_ctx();
    h->ns = ns; h->M = 2 * ns; h->nu = nu; h->nd = nd; h->N = N; h->ncorr = ans->n_corr;
    h->P = nu * (nu - 1) / 2 + nd * (nd - 1) / 2 + nu * nd;
    h->npf = h->M * (h->M - 1) / 2;
    h->n_walkers = opt->n_walkers;
    h->spw = opt->samples_per_walker;
    h->ncap = (int64_t)opt->n_walkers * opt->samples_per_walker;
    h->wprec = opt->walker_precision;
    h->keep64 = opt->keep_fp64_store ? 1 : 0;
    h->keeplow = opt->keep_lowp_store ? 1 : 0;
    h->refresh_every = opt->refresh_every > 0 ? opt->refresh_every : 0;
    h->fp64_refresh = (opt->fp64_refresh && opt->walker_precision == VMC_FP32) ? 1 : 0;
    h->ham = ham->kind;
    auto fail = [&](int code) { vmc_destroy(h); return code; };
    if (h->ncap > (int64_t)1 << 31) return fail(VMC_ERR_INVALID_ARG);
    if (!h->keep64 && !h->keeplow) return fail(VMC_ERR_INVALID_ARG);

    // correlators
    std::vector<int> cptr(h->ncorr + 1, 0), csites;
    h->corr_off.assign(h->ncorr + 1, 0);
    std::vector<std::vector<std::pair<int, int>>> memb(ns);
    for (int c = 0; c < h->ncorr; ++c) {
        int b = ans->corr_ptr[c], e = ans->corr_ptr[c + 1];
        int m = e - b;
        if (m < 1 || m > 9) return fail(VMC_ERR_INVALID_ARG);
        int w = 1;
        for (int j = b; j < e; ++j) {
            int s = ans->corr_sites[j];
            if (s < 0 || s >= ns) return fail(VMC_ERR_INVALID_ARG);
            for (int j2 = b; j2 < j; ++j2)
                if (ans->corr_sites[j2] == s) return fail(VMC_ERR_INVALID_ARG);
            csites.push_back(s);
            memb[s].push_back({c, w});
            w *= 4;
        }
        cptr[c + 1] = (int)csites.size();
        h->maxd = std::max(h->maxd, 1 << (2 * m));
    }
    // classes: correlators of one class share one parameter block; blocks in
    // class order, corr_off[c] = first parameter of c's block
    std::vector<int> cls(h->ncorr);
    for (int c = 0; c < h->ncorr; ++c) cls[c] = ans->corr_class ? ans->corr_class[c] : c;
    h->n_class = 0;
    for (int c = 0; c < h->ncorr; ++c) {
        if (cls[c] < 0 || cls[c] >= h->ncorr) return fail(VMC_ERR_INVALID_ARG);
        h->n_class = std::max(h->n_class, cls[c] + 1);
    }
    std::vector<int> cm(h->n_class, 0);
    for (int c = 0; c < h->ncorr; ++c) {
        const int m = cptr[c + 1] - cptr[c];
        if (cm[cls[c]] != 0 && cm[cls[c]] != m) return fail(VMC_ERR_INVALID_ARG);   // one size per class
        cm[cls[c]] = m;
    }
    std::vector<int64_t> class_off(h->n_class + 1, 0);
    for (int q = 0; q < h->n_class; ++q) {
        if (cm[q] == 0) return fail(VMC_ERR_INVALID_ARG);                             // unused class id
        class_off[q + 1] = class_off[q] + ((int64_t)1 << (2 * cm[q]));
    }
    std::vector<int> class_ptr(h->n_class + 1, 0), class_inst;
    for (int q = 0; q < h->n_class; ++q) {
        for (int c = 0; c < h->ncorr; ++c)
            if (cls[c] == q) class_inst.push_back(c);
        class_ptr[q + 1] = (int)class_inst.size();
    }
    // histogram-scatter work units: up to kInstPerUnit correlators of one class
    std::vector<int4> units;
    for (int q = 0; q < h->n_class; ++q)
        for (int j = class_ptr[q]; j < class_ptr[q + 1]; j += kInstPerUnit)
            units.push_back(make_int4(q, j, std::min(j + kInstPerUnit, class_ptr[q + 1]), 0));
    h->n_units = (int)units.size();
    h->corr_off.assign(h->ncorr + 1, 0);
    for (int c = 0; c < h->ncorr; ++c) h->corr_off[c] = class_off[cls[c]];
    h->ncp = class_off[h->n_class];
    h->corr_off[h->ncorr] = h->ncp;
    h->nv = h->ncp + h->npf;
    // dense (correlator, site) -> 4^j weight table, 0 where the site is absent
    std::vector<uint32_t> csw((size_t)std::max(h->ncorr, 1) * ns, 0);
    for (int s = 0; s < ns; ++s)
        for (auto& pr : memb[s]) csw[(size_t)pr.first * ns + s] = (uint32_t)pr.second;
    std::vector<int> scptr(ns + 1, 0), scorr, sw;
    for (int s = 0; s < ns; ++s) {
        for (auto& pr : memb[s]) { scorr.push_back(pr.first); sw.push_back(pr.second); }
        scptr[s + 1] = (int)scorr.size();
    }
    // hopping lists (each bond hops both ways; repeated bonds repeat)
    std::vector<std::vector<std::pair<int, double>>> nb(ns);
    for (int b = 0; b < lat->n_bonds; ++b) {
        int i = lat->bonds[2 * b], j = lat->bonds[2 * b + 1];
        if (i < 0 || j < 0 || i >= ns || j >= ns) return fail(VMC_ERR_INVALID_ARG);
        if (i == j) continue;
        nb[i].push_back({j, lat->bond_t[b]});
        nb[j].push_back({i, lat->bond_t[b]});
    }
    std::vector<int> nptr(ns + 1, 0), nsite;
    std::vector<double> nt;
    for (int s = 0; s < ns; ++s) {
        for (auto& pr : nb[s]) { nsite.push_back(pr.first); nt.push_back(pr.second); }
        nptr[s + 1] = (int)nsite.size();
    }
    // correlators containing both sites i and j (i != j)
    h->max_csites = 0;
    for (int c = 0; c < h->ncorr; ++c) h->max_csites = std::max(h->max_csites, cptr[c + 1] - cptr[c]);
    std::vector<int> pptr((size_t)ns * ns + 1, 0), pcorr;
    {
        std::vector<std::vector<int>> pl((size_t)ns * ns);
        for (int c = 0; c < h->ncorr; ++c)
            for (int j1 = cptr[c]; j1 < cptr[c + 1]; ++j1)
                for (int j2 = cptr[c]; j2 < cptr[c + 1]; ++j2)
                    if (j1 != j2) pl[(size_t)csites[j1] * ns + csites[j2]].push_back(c);
        h->pair_unique = h->ncp < ((int64_t)1 << 30);
        for (size_t k = 0; k < pl.size(); ++k) {
            for (int c : pl[k]) pcorr.push_back(c);
            pptr[k + 1] = (int)pcorr.size();
            if (pl[k].size() > 1) h->pair_unique = false;
        }
    }
    // ab initio integrals: (pq|rs) = sum_mu L^mu_pq L^mu_rs (Eq. 9 with R = L)
    std::vector<double> eri64, h64;
    if (ham->kind == VMC_ABINITIO) {
        const size_t n2 = (size_t)ns * ns;
        h64.assign(ham->h, ham->h + n2);
        eri64.assign(n2 * n2, 0.0);
        for (int mu = 0; mu < ham->n_chol; ++mu) {
            const double* L = ham->chol + (size_t)mu * n2;
            for (size_t pq = 0; pq < n2; ++pq) {
                const double l = L[pq];
                if (l == 0.0) continue;
                double* row = eri64.data() + pq * n2;
                for (size_t rs = 0; rs < n2; ++rs) row[rs] += l * L[rs];
            }
        }
    }
    // Eq. 9 factors for the linear method.  A one-body K = sum k_ij E_ij
    // (E_ij = sum_s a+_is a_js) commutes with the particle number, so in the
    // N-electron sector K = (K Nhat + Nhat K) / 2N: the pairs (k/2N, I) and
    // (I, k/2N).  Hubbard: k = -t per bond and direction; U n_up n_dn =
    // (U/2)(E_ii E_ii - E_ii): (U/2 e_i e_i^T, e_i e_i^T) per site and the
    // constant -U N / 2.  Ab initio: a+_p a+_r a_s a_q = E_pq E_rs - delta_qr
    // E_ps, so the pairs (L^mu/sqrt2, L^mu/sqrt2) and k = h - J/2 with
    // J_ps = sum_q (pq|qs).
    {
        const size_t n2 = (size_t)ns * ns;
        std::vector<double> k(n2, 0.0);
        auto push = [&](const std::vector<double>& L, const std::vector<double>& R) {
            h->lm_L.insert(h->lm_L.end(), L.begin(), L.end());
            h->lm_R.insert(h->lm_R.end(), R.begin(), R.end());
            h->lm_nmu++;
        };
        if (ham->kind == VMC_HUBBARD) {
            for (int i = 0; i < ns; ++i)
                for (auto& pr : nb[i]) k[(size_t)i * ns + pr.first] -= pr.second;
            for (int i = 0; i < ns; ++i) {
                std::vector<double> L(n2, 0.0), R(n2, 0.0);
                L[(size_t)i * ns + i] = 0.5 * ham->U;
                R[(size_t)i * ns + i] = 1.0;
                push(L, R);
            }
            h->lm_c0 = -0.5 * ham->U * N;
        } else {
            std::vector<double> J(n2, 0.0);
            for (int mu = 0; mu < ham->n_chol; ++mu) {
                const double* L = ham->chol + (size_t)mu * n2;
                for (int p = 0; p < ns; ++p)
                    for (int q = 0; q < ns; ++q)
                        for (int r = 0; r < ns; ++r) J[(size_t)p * ns + r] += L[(size_t)p * ns + q] * L[(size_t)q * ns + r];
                std::vector<double> Ls(L, L + n2);
                for (auto& v : Ls) v *= std::sqrt(0.5);
                push(Ls, Ls);
            }
            for (size_t t = 0; t < n2; ++t) k[t] = ham->h[t] - 0.5 * J[t];
        }
        std::vector<double> I(n2, 0.0), kh(n2);
        for (int i = 0; i < ns; ++i) I[(size_t)i * ns + i] = 1.0;
        for (size_t t = 0; t < n2; ++t) kh[t] = k[t] / (2.0 * N);
        push(kh, I);
        push(I, kh);
    }
    // pairing block order: up-up triangle, down-down triangle, up-down rectangle
    std::vector<uint16_t> pt;
    for (int a = 0; a < nu; ++a)
        for (int b = a + 1; b < nu; ++b) pt.push_back((uint16_t)(a | (b << 8)));
    for (int a = nu; a < N; ++a)
        for (int b = a + 1; b < N; ++b) pt.push_back((uint16_t)(a | (b << 8)));
    for (int a = 0; a < nu; ++a)
        for (int b = nu; b < N; ++b) pt.push_back((uint16_t)(a | (b << 8)));
    std::vector<int> rb(h->M);
    for (int p = 0; p < h->M; ++p) rb[p] = (int)pf_row_base(h->M, p);
    std::vector<uint32_t> pqo((size_t)h->M * (h->M - 1) / 2);
    for (int p = 0; p < h->M; ++p)
        for (int q = p + 1; q < h->M; ++q) pqo[(size_t)rb[p] + q] = (uint32_t)p | ((uint32_t)q << 16);

    if (cudaGetDevice(&h->dev) != cudaSuccess) return fail(VMC_ERR_CUDA);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->dev) != cudaSuccess) return fail(VMC_ERR_CUDA);
    h->nsm = prop.multiProcessorCount;
    h->smem_optin = prop.sharedMemPerBlockOptin;
    h->coop_launch = prop.cooperativeLaunch != 0;

#define ACK(x) do { if ((x) != cudaSuccess) { set_err(#x); return fail(VMC_ERR_OOM); } } while (0)
#define UPL(dst, src, n) do { if (cudaMemcpy(dst, src, sizeof(*(dst)) * (n), cudaMemcpyHostToDevice) != cudaSuccess) return fail(VMC_ERR_CUDA); } while (0)
    ACK(h->alloc(&h->d_corr_ptr, cptr.size()));
    ACK(h->alloc(&h->d_corr_sites, csites.size()));
    ACK(h->alloc(&h->d_corr_off, h->corr_off.size()));
    ACK(h->alloc(&h->d_class_off, class_off.size()));
    ACK(h->alloc(&h->d_class_ptr, class_ptr.size()));
    ACK(h->alloc(&h->d_class_inst, std::max<size_t>(class_inst.size(), 1)));
    ACK(h->alloc(&h->d_units, std::max<size_t>(units.size(), 1)));
    ACK(h->alloc(&h->d_site_cptr, scptr.size()));
    ACK(h->alloc(&h->d_site_corr, scorr.size()));
    ACK(h->alloc(&h->d_site_w, sw.size()));
    ACK(h->alloc(&h->d_corr_site_w, csw.size()));
    ACK(h->alloc(&h->d_nbr_ptr, nptr.size()));
    ACK(h->alloc(&h->d_nbr_site, nsite.size()));
    ACK(h->alloc(&h->d_nbr_t, nt.size()));
    ACK(h->alloc(&h->d_pairtab, pt.size()));
    ACK(h->alloc(&h->d_rowbase, rb.size()));
    ACK(h->alloc(&h->d_pq_of, std::max<size_t>(pqo.size(), 1)));
    UPL(h->d_corr_ptr, cptr.data(), cptr.size());
    if (!csites.empty()) UPL(h->d_corr_sites, csites.data(), csites.size());
    UPL(h->d_corr_off, h->corr_off.data(), h->corr_off.size());
    UPL(h->d_class_off, class_off.data(), class_off.size());
    UPL(h->d_class_ptr, class_ptr.data(), class_ptr.size());
    if (!class_inst.empty()) UPL(h->d_class_inst, class_inst.data(), class_inst.size());
    if (!units.empty()) UPL(h->d_units, units.data(), units.size());
    UPL(h->d_site_cptr, scptr.data(), scptr.size());
    if (!scorr.empty()) UPL(h->d_site_corr, scorr.data(), scorr.size());
    if (!sw.empty()) UPL(h->d_site_w, sw.data(), sw.size());
    UPL(h->d_corr_site_w, csw.data(), csw.size());
    UPL(h->d_nbr_ptr, nptr.data(), nptr.size());
    if (!nsite.empty()) UPL(h->d_nbr_site, nsite.data(), nsite.size());
    if (!nt.empty()) UPL(h->d_nbr_t, nt.data(), nt.size());
    UPL(h->d_pairtab, pt.data(), pt.size());
    UPL(h->d_rowbase, rb.data(), rb.size());
    if (!pqo.empty()) UPL(h->d_pq_of, pqo.data(), pqo.size());
    ACK(h->alloc(&h->d_pair_ptr, pptr.size()));
    ACK(h->alloc(&h->d_pair_corr, std::max<size_t>(pcorr.size(), 1)));
    UPL(h->d_pair_ptr, pptr.data(), pptr.size());
    if (!pcorr.empty()) UPL(h->d_pair_corr, pcorr.data(), pcorr.size());
    if (ham->kind == VMC_ABINITIO) {
        std::vector<float> h32(h64.begin(), h64.end()), eri32(eri64.begin(), eri64.end());
        ACK(h->alloc(&h->d_h64, h64.size()));
        ACK(h->alloc(&h->d_h32, h32.size()));
        ACK(h->alloc(&h->d_eri64, eri64.size()));
        ACK(h->alloc(&h->d_eri32, eri32.size()));
        UPL(h->d_h64, h64.data(), h64.size());
        UPL(h->d_h32, h32.data(), h32.size());
        UPL(h->d_eri64, eri64.data(), eri64.size());
        UPL(h->d_eri32, eri32.data(), eri32.size());
        // double excitations: electron-position pairs, then empty-orbital
        // index pairs, of the up-up, down-down and up-down classes
        const int eu = ns - nu, ed = ns - nd;
        std::vector<uint16_t> dx;
        for (int a = 0; a < nu; ++a)
            for (int b = a + 1; b < nu; ++b) dx.push_back((uint16_t)(a | b << 8));
        for (int a = nu; a < N; ++a)
            for (int b = a + 1; b < N; ++b) dx.push_back((uint16_t)(a | b << 8));
        for (int a = 0; a < nu; ++a)
            for (int b = nu; b < N; ++b) dx.push_back((uint16_t)(a | b << 8));
        for (int x = 0; x < eu; ++x)
            for (int y = x + 1; y < eu; ++y) dx.push_back((uint16_t)(x | y << 8));
        for (int x = eu; x < eu + ed; ++x)
            for (int y = x + 1; y < eu + ed; ++y) dx.push_back((uint16_t)(x | y << 8));
        for (int x = 0; x < eu; ++x)
            for (int y = eu; y < eu + ed; ++y) dx.push_back((uint16_t)(x | y << 8));
        ACK(h->alloc(&h->d_dexc, std::max<size_t>(dx.size(), 1)));
        if (!dx.empty()) UPL(h->d_dexc, dx.data(), dx.size());
    }
    // parameters
    ACK(h->alloc(&h->d_C64, h->ncp));
    ACK(h->alloc(&h->d_invC64, h->ncp));
    ACK(h->alloc(&h->d_C32, h->ncp));
    ACK(h->alloc(&h->d_invC32, h->ncp));
    ACK(h->alloc(&h->d_F64, (size_t)h->M * h->M));
    ACK(h->alloc(&h->d_F32, (size_t)h->M * h->M));
    // walkers
    ACK(h->alloc(&h->d_wocc, (size_t)h->n_walkers * N));
    ACK(h->alloc(&h->d_wstep, h->n_walkers));
    ACK(h->alloc(&h->d_mocc, (size_t)h->ncap * N));
    // O store
    h->Nst = (int)round_up(N, 16);
    h->ncst = (int)round_up(std::max(h->ncorr, 1), 8);
    h->Pst = round_up(h->P, 8);
    ACK(h->alloc(&h->d_socc, (size_t)h->ncap * h->Nst));
    ACK(h->alloc(&h->d_cidx, (size_t)h->ncap * h->ncst));
    ACK(h->alloc(&h->d_cidxT, (size_t)h->ncap * std::max(h->ncorr, 1)));
    ACK(h->alloc(&h->d_E, h->ncap));
    ACK(h->alloc(&h->d_lnrun, h->ncap));
    if (h->fp64_refresh) ACK(h->alloc(&h->d_Echain, h->ncap));
    if (h->keep64) ACK(h->alloc(&h->d_pf64, (size_t)h->ncap * h->Pst));
    if (h->keeplow) {
        ACK(h->alloc(&h->d_pf32, (size_t)h->ncap * h->Pst));
        ACK(h->alloc(&h->d_pf16, (size_t)h->ncap * h->Pst));
        // sorted two-pass structures for the BF16 product
        h->sort_nblk = 2 * h->nsm;
        h->sort_nchunk = (int)((h->ncap + kTChunk - 1) / kTChunk);
        {
            const int QE = (h->P + kGParts - 1) / kGParts;
            h->gwq = (QE + 3) / 4;
            h->Gst = (int64_t)kGParts * h->gwq * 4;
            std::vector<uint32_t> ft;
            const int Puu = nu * (nu - 1) / 2, Pdd = nd * (nd - 1) / 2;
            for (int a = 0; a < N; ++a)
                for (int b = a + 1; b < N; ++b) {
                    int e;
                    if (b < nu) e = a * nu - a * (a + 1) / 2 + (b - a - 1);
                    else if (a >= nu) e = Puu + (a - nu) * nd - (a - nu) * (a - nu + 1) / 2 + (b - a - 1);
                    else e = Puu + Pdd + a * nd + (b - nu);
                    ft.push_back((uint32_t)e | ((uint32_t)a << 16) | ((uint32_t)b << 24));
                }
            ACK(h->alloc(&h->d_fulltab, std::max<size_t>(ft.size(), 1)));
            if (!ft.empty() && cudaMemcpy(h->d_fulltab, ft.data(), sizeof(uint32_t) * ft.size(),
                                          cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(VMC_ERR_CUDA);
        }
        ACK(h->alloc(&h->d_G, (size_t)h->ncap * h->Gst));
        // compact copy: the values of each row in the row-major pair order,
        // rows padded to 16 bytes, and the pair of each 16-byte word's first value
        h->Gst16 = round_up(h->P, 8);
        if (N <= 255) {
            ACK(h->alloc(&h->d_G16, (size_t)h->ncap * h->Gst16));
            std::vector<uint16_t> wt((size_t)(h->Gst16 / 8));
            int a = 0, b = 1;
            for (int64_t r = 0; r < h->Gst16; ++r) {
                if (r % 8 == 0) wt[(size_t)(r / 8)] = r < h->P ? (uint16_t)(a | b << 8) : (uint16_t)((N - 1) | N << 8);
                if (++b == N) { ++a; b = a + 1; }
            }
            ACK(h->alloc(&h->d_wtab, wt.size()));
            if (cudaMemcpy(h->d_wtab, wt.data(), sizeof(uint16_t) * wt.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                return fail(VMC_ERR_CUDA);
        }
        h->t_chunk = (size_t)kTChunk * h->P + (size_t)h->npf * kTRun;   // padded runs of one chunk
        ACK(h->alloc(&h->d_Tsort, (size_t)h->sort_nchunk * h->t_chunk));
        if (h->sort_nchunk > 1) ACK(h->alloc(&h->d_tpart, (size_t)h->sort_nchunk * h->npf * kMaxK));
        ACK(h->alloc(&h->d_tdone, (size_t)h->npf));
        if (cudaMemset(h->d_tdone, 0, sizeof(unsigned) * h->npf) != cudaSuccess) return fail(VMC_ERR_CUDA);
        ACK(h->alloc(&h->d_counts, (size_t)h->sort_nblk * h->npf));
        ACK(h->alloc(&h->d_total, (size_t)h->npf));
        ACK(h->alloc(&h->d_base, (size_t)h->sort_nchunk * (h->npf + 1)));
        ACK(h->alloc(&h->d_Tc, (size_t)h->ncap * std::max(h->ncorr, 1)));
        ACK(h->alloc(&h->d_ccount, (size_t)std::max<int64_t>(h->ncp, 1)));
        ACK(h->alloc(&h->d_cbase, (size_t)h->ncp + 1));
        const int64_t ng = (h->ncp + 31) / 32;
        h->max_items = ng + (h->ncap * std::max(h->ncorr, 1) + kCorrItem - 1) / kCorrItem;
        ACK(h->alloc(&h->d_items, (size_t)std::max<int64_t>(h->max_items, 1)));
        ACK(h->alloc(&h->d_nitems, (size_t)std::max<int64_t>(ng, 1)));
        ACK(h->alloc(&h->d_item_base, (size_t)ng + 1));
    }
    for (int k = 0; k < 3; ++k) ACK(h->alloc(&h->d_Obar[k], h->nv));
    for (int k = 0; k < 3; ++k) ACK(h->alloc(&h->d_Obar32[k], h->nv));
    ACK(h->alloc(&h->d_status, 4));
    // scratch
    ACK(h->alloc((double**)&h->d_T, (size_t)h->ncap * kMaxK));
    h->pfpart_bytes = (size_t)4 * h->nsm * h->npf * kMaxK * sizeof(double);
    ACK(h->alloc((char**)&h->d_pfpart, h->pfpart_bytes));
    ACK(h->alloc(&h->d_corrraw, (size_t)std::max<int64_t>(h->ncp, 1) * kMaxK));
    ACK(h->alloc(&h->d_part, (size_t)8 * kNumPart * kMaxK));
    ACK(h->alloc(&h->d_pfraw, (size_t)h->npf * kMaxK));
    ACK(h->alloc(&h->d_scal, 16));
    ACK(h->alloc(&h->d_stop, 4));
    const size_t vk = (size_t)h->nv * kMaxK;
    ACK(h->alloc(&h->d_x64, vk)); ACK(h->alloc(&h->d_r64, vk)); ACK(h->alloc(&h->d_p64, vk));
    ACK(h->alloc(&h->d_q64, vk)); ACK(h->alloc(&h->d_t64, vk));
    ACK(h->alloc(&h->d_x32, vk)); ACK(h->alloc(&h->d_r32, vk)); ACK(h->alloc(&h->d_p32, vk));
    ACK(h->alloc(&h->d_q32, vk)); ACK(h->alloc(&h->d_b32, vk));
    if (cudaMallocHost((void**)&h->h_pinned, 64 * sizeof(double)) != cudaSuccess) return fail(VMC_ERR_OOM);
    if (cudaMemset(h->d_status, 0, 4 * sizeof(int)) != cudaSuccess) return fail(VMC_ERR_CUDA);
    if (cudaMemset(h->d_wstep, 0, sizeof(uint64_t) * h->n_walkers) != cudaSuccess) return fail(VMC_ERR_CUDA);
#undef ACK
#undef UPL

    DevProblem& pb = h->pb;
    pb.ns = ns; pb.M = h->M; pb.nu = nu; pb.nd = nd; pb.N = N; pb.ncorr = h->ncorr; pb.P = h->P;
    pb.npf = h->npf; pb.ham = h->ham; pb.ncp = h->ncp; pb.nv = h->nv; pb.U = ham->U;
    pb.corr_ptr = h->d_corr_ptr; pb.corr_sites = h->d_corr_sites; pb.corr_off = h->d_corr_off;
    pb.n_class = h->n_class; pb.class_off = h->d_class_off;
    pb.class_ptr = h->d_class_ptr; pb.class_inst = h->d_class_inst;
    pb.site_cptr = h->d_site_cptr; pb.site_corr = h->d_site_corr; pb.site_w = h->d_site_w;
    pb.corr_site_w = h->d_corr_site_w;
    pb.nbr_ptr = h->d_nbr_ptr; pb.nbr_site = h->d_nbr_site; pb.nbr_t = h->d_nbr_t;
    pb.h64 = h->d_h64; pb.h32 = h->d_h32; pb.eri64 = h->d_eri64; pb.eri32 = h->d_eri32;
    pb.pair_ptr = h->d_pair_ptr; pb.pair_corr = h->d_pair_corr;
    pb.pair_unique = h->pair_unique ? 1 : 0;
    pb.dexc = h->d_dexc;
    pb.max_csites = h->max_csites;
    pb.ff_sums = h->ff_sums ? 1 : 0;
    pb.C64 = h->d_C64; pb.C32 = h->d_C32; pb.F64 = h->d_F64; pb.F32 = h->d_F32;
    pb.pairtab = h->d_pairtab; pb.rowbase = h->d_rowbase;
    *out = h;
    return VMC_OK;
}

extern "C" int vmc_destroy(vmc_handle h) {
    if (!h) return VMC_OK;
    for (auto& r : h->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    for (void* p : h->allocs) cudaFree(p);
    if (h->h_pinned) cudaFreeHost(h->h_pinned);
    delete h;
    return VMC_OK;
}

extern "C" int vmc_num_params(vmc_handle h, int64_t* n_v, int64_t* n_corr_params) {
    if (!h) return VMC_ERR_INVALID_ARG;
    if (n_v) *n_v = h->nv;
    if (n_corr_params) *n_corr_params = h->ncp;
    return VMC_OK;
}

extern "C" int vmc_num_samples(vmc_handle h, int64_t* n_s) {
    if (!h || !n_s) return VMC_ERR_INVALID_ARG;
    *n_s = h->n_s;
    return VMC_OK;
}

extern "C" int vmc_set_params(vmc_handle h, const double* C, const double* f) {
    if (!h || (!C && h->ncp > 0) || !f) return VMC_ERR_INVALID_ARG;
    const int M = h->M;
    std::vector<double> c64(C, C + h->ncp), ic64(h->ncp), F64((size_t)M * M, 0.0);
    std::vector<float> c32(h->ncp), ic32(h->ncp), F32((size_t)M * M, 0.f);
    for (int64_t k = 0; k < h->ncp; ++k) {
        if (C[k] == 0.0 || !std::isfinite(C[k])) return VMC_ERR_SINGULAR;
        ic64[k] = 1.0 / C[k];
        c32[k] = (float)C[k];
        ic32[k] = (float)ic64[k];
    }
    for (int p = 0; p < M; ++p)
        for (int q = p + 1; q < M; ++q) {
            double v = f[pf_row_base(M, p) + q];
            if (!std::isfinite(v)) return VMC_ERR_NONFINITE;
            F64[(size_t)p * M + q] = v;
            F64[(size_t)q * M + p] = -v;
            F32[(size_t)p * M + q] = (float)v;
            F32[(size_t)q * M + p] = -(float)v;
        }
    // the copies below overwrite buffers that kernels queued on any stream
    // may still read: wait for all work on the device first
    VCK(cudaDeviceSynchronize());
    VCK(cudaMemcpy(h->d_C64, c64.data(), sizeof(double) * h->ncp, cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(h->d_invC64, ic64.data(), sizeof(double) * h->ncp, cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(h->d_C32, c32.data(), sizeof(float) * h->ncp, cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(h->d_invC32, ic32.data(), sizeof(float) * h->ncp, cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(h->d_F64, F64.data(), sizeof(double) * M * M, cudaMemcpyHostToDevice));
    VCK(cudaMemcpy(h->d_F32, F32.data(), sizeof(float) * M * M, cudaMemcpyHostToDevice));
    h->params_set = true;
    h->obar_ok[0] = h->obar_ok[1] = h->obar_ok[2] = false;
    h->sorted_ok = h->g_ok = h->corr_ok = false;
    return VMC_OK;
}

extern "C" int vmc_get_params(vmc_handle h, double* C, double* f, void* stream) {
    if (!h) return VMC_ERR_INVALID_ARG;
    if (!h->params_set) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    const int M = h->M;
    std::vector<double> F64;
    if (C && h->ncp > 0) VCK(cudaMemcpyAsync(C, h->d_C64, sizeof(double) * h->ncp, cudaMemcpyDeviceToHost, st));
    if (f) {
        F64.resize((size_t)M * M);
        VCK(cudaMemcpyAsync(F64.data(), h->d_F64, sizeof(double) * M * M, cudaMemcpyDeviceToHost, st));
    }
    VCK(cudaStreamSynchronize(st));
    if (f)
        for (int p = 0; p < M; ++p)
            for (int q = p + 1; q < M; ++q) f[pf_row_base(M, p) + q] = F64[(size_t)p * M + q];
    return VMC_OK;
}

static int check_configs(const vmc_ctx* h, const uint8_t* occ, int64_t n) {
    for (int64_t w = 0; w < n; ++w) {
        const uint8_t* o = occ + w * h->N;
        for (int a = 0; a < h->N; ++a) {
            if (o[a] >= h->M) return VMC_ERR_INVALID_ARG;
            if (a > 0 && o[a] <= o[a - 1]) return VMC_ERR_INVALID_ARG;
            if ((a < h->nu) != (o[a] < h->ns)) return VMC_ERR_INVALID_ARG;
        }
    }
    return VMC_OK;
}

extern "C" int vmc_set_walkers(vmc_handle h, const uint8_t* occ, const uint64_t* step) {
    if (!h || !occ) return VMC_ERR_INVALID_ARG;
    int rc = check_configs(h, occ, h->n_walkers);
    if (rc) return rc;
    VCK(cudaDeviceSynchronize());   // a sampling call on any stream may still use the walkers
    VCK(cudaMemcpy(h->d_wocc, occ, (size_t)h->n_walkers * h->N, cudaMemcpyHostToDevice));
    if (step) VCK(cudaMemcpy(h->d_wstep, step, sizeof(uint64_t) * h->n_walkers, cudaMemcpyHostToDevice));
    else VCK(cudaMemset(h->d_wstep, 0, sizeof(uint64_t) * h->n_walkers));
    h->walkers_set = true;
    return VMC_OK;
}

extern "C" int vmc_get_walkers(vmc_handle h, uint8_t* occ, uint64_t* step, void* stream) {
    if (!h) return VMC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    VCK(cudaStreamSynchronize(st));
    if (occ) VCK(cudaMemcpy(occ, h->d_wocc, (size_t)h->n_walkers * h->N, cudaMemcpyDeviceToHost));
    if (step) VCK(cudaMemcpy(step, h->d_wstep, sizeof(uint64_t) * h->n_walkers, cudaMemcpyDeviceToHost));
    return VMC_OK;
}

// ---------------------------------------------------------------------------
// walker kernels
// ---------------------------------------------------------------------------
static int read_status(vmc_ctx* h, cudaStream_t st) {
    int s = 0;
    VCK(cudaMemcpyAsync(h->h_pinned, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    VCK(cudaStreamSynchronize(st));
    memcpy(&s, h->h_pinned, sizeof(int));
    VCK(cudaMemsetAsync(h->d_status, 0, sizeof(int), st));
    if (s & ST_BAD_CONFIG) return VMC_ERR_INVALID_ARG;
    if (s & ST_SINGULAR) return VMC_ERR_SINGULAR;
    if (s & ST_NONFINITE) return VMC_ERR_NONFINITE;
    if (s & ST_TIMEOUT) return VMC_ERR_TIMEOUT;
    return VMC_OK;
}

// fills the problem-dependent fields of `a` (strides, shared-memory slice per
// walker) and returns the slice size
static size_t prep_walkers(vmc_ctx* h, SampleArgs& a, bool fp64) {
    a.pb = h->pb;
    a.XS = (h->N + 2) & ~1;   // even (the rank-2 update moves column pairs), N + 1 or N + 2
    a.GS = h->N + 1;
    a.ncorr_pad = (int)round_up(std::max(h->ncorr, 1), 4);
    const size_t rsz = fp64 ? 8 : 4;
    size_t wb = (size_t)h->N * a.XS * rsz + 3 * (size_t)a.XS * rsz;
    wb = wb + 64 + (size_t)a.ncorr_pad * 4 + 64 + 128;
    if (h->ham == VMC_ABINITIO && a.want_energy) {
        // G [M][GS], H [E][E], single-move factors [N][E], empty list, index
        // map, per-site factors [ns][4]
        const size_t E = (size_t)(h->M - h->N);
        wb += ((size_t)h->M * a.GS + E * E + (size_t)h->N * E) * rsz + 128 + 128 + (size_t)4 * h->ns * rsz;
        // the sample's site-pair table (pair correlators, each pair in at most one)
        if (h->max_csites <= 2 && h->pair_unique) wb += (size_t)h->ns * (h->ns - 1) / 2 * 4;
    }
    wb = round_up(wb, 16);
    a.warp_bytes = wb;
    a.status = h->d_status;
    return wb;
}

static int launch_walkers(vmc_ctx* h, SampleArgs& a, bool fp64, cudaStream_t st) {
    const size_t wb = prep_walkers(h, a, fp64);
    int wpb = (int)std::min<size_t>(4, h->smem_optin / wb);
    if (wpb < 1) return VMC_ERR_UNSUPPORTED;
    size_t smem = wb * wpb;
    int blocks = (a.n_walkers + wpb - 1) / wpb;
    if (fp64) {
        VCK(cudaFuncSetAttribute(k_walkers<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_walkers<double><<<blocks, 32 * wpb, smem, st>>>(a); h->n_launch++;
    } else {
        VCK(cudaFuncSetAttribute(k_walkers<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        // shared-memory carveout (percent of the maximum): the ab initio local
        // energy reads integral, correlator and pair tables through L1
        VCK(cudaFuncSetAttribute(k_walkers<float>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 h->ham == VMC_ABINITIO ? h->walker_carveout_ab : -1));
        k_walkers<float><<<blocks, 32 * wpb, smem, st>>>(a); h->n_launch++;
    }
    VCK(cudaGetLastError());
    return VMC_OK;
}

static void store_targets(vmc_ctx* h, SampleArgs& a) {
    a.s_occ = h->d_socc; a.Nst = h->Nst;
    a.s_cidx = h->d_cidx; a.ncst = h->ncst;
    a.s_E = h->d_E;
    a.s_lnrun = h->d_lnrun;
    a.s_pf64 = h->keep64 ? h->d_pf64 : nullptr;
    a.s_pf32 = h->keeplow ? h->d_pf32 : nullptr;
    a.s_pf16 = h->keeplow ? h->d_pf16 : nullptr;
    a.Pst = h->Pst;
}

static int transpose_states(vmc_ctx* h, cudaStream_t st) {
    if (h->ncorr == 0 || h->n_s == 0) return VMC_OK;
    dim3 grid((unsigned)((h->n_s + 31) / 32), (unsigned)((h->ncorr + 31) / 32));
    k_transpose_cidx<<<grid, 256, 0, st>>>(h->d_cidx, h->ncst, h->ncorr, h->n_s, h->d_cidxT); h->n_launch++;
    VCK(cudaGetLastError());
    return VMC_OK;
}

static void sample_args(vmc_ctx* h, int n_burn, uint64_t seed, SampleArgs& a) {
    a = SampleArgs{};
    a.n_walkers = h->n_walkers;
    a.spw = h->spw;
    a.n_burn = n_burn;
    a.props_per_sweep = h->N;
    a.write_back = 1;
    a.refresh_every = h->refresh_every;
    a.want_energy = 1;
    a.seed = seed;
    a.walker_occ = h->d_wocc;
    a.walker_step = h->d_wstep;
    store_targets(h, a);
}

static int after_sampling(vmc_ctx* h, cudaStream_t st);

extern "C" int vmc_sample(vmc_handle h, int n_burn, uint64_t seed, void* stream) {
    if (!h || n_burn < 0) return VMC_ERR_INVALID_ARG;
    if (!h->params_set || !h->walkers_set) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    SampleArgs a;
    sample_args(h, n_burn, seed, a);
    int rc = launch_walkers(h, a, h->wprec == VMC_FP64, st);
    if (rc) return rc;
    return after_sampling(h, st);
}

// the store holds a new set of samples: invalidate what was built on the old
// one, refresh in FP64 if asked, transpose the correlator states
static int after_sampling(vmc_ctx* h, cudaStream_t st) {
    int rc;
    h->n_s = h->ncap;
    h->obar_ok[0] = h->obar_ok[1] = h->obar_ok[2] = false;
    h->sorted_ok = h->g_ok = h->corr_ok = false;
    h->refreshed = false;
    if (h->wprec == VMC_FP32 && h->fp64_refresh) {
        // FP64 refresh of every stored sample: the pairing inverse, E_L and O
        // from scratch in FP64, rounded into the stores; the chains' own E_L
        // is kept for the statistics
        VCK(cudaMemcpyAsync(h->d_Echain, h->d_E, sizeof(double) * h->n_s, cudaMemcpyDeviceToDevice, st));
        VCK(cudaMemcpy2DAsync(h->d_mocc, h->N, h->d_socc, h->Nst, h->N, h->n_s, cudaMemcpyDeviceToDevice, st));
        SampleArgs m{};
        m.n_walkers = (int)h->n_s;
        m.spw = 1;
        m.want_energy = 1;
        m.walker_occ = h->d_mocc;
        store_targets(h, m);
        m.s_lnrun = nullptr;   // keep the chains' running log-amplitudes
        rc = launch_walkers(h, m, true, st);
        if (rc) return rc;
        h->refreshed = true;
    }
    rc = transpose_states(h, st);
    if (rc) return rc;
    return read_status(h, st);
}

// device buffer for the argument blocks of the batched launches
static int batch_buffer(vmc_ctx* h, size_t bytes, void** p) {
    if (h->batch_bytes < bytes) {
        if (h->d_batch) {
            cudaFree(h->d_batch);
            h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), h->d_batch));
            h->d_batch = nullptr;
        }
        unsigned char* q = nullptr;
        VCK(h->alloc(&q, bytes));
        h->d_batch = q;
        h->batch_bytes = bytes;
    }
    *p = h->d_batch;
    return VMC_OK;
}

extern "C" int vmc_sample_batch(const vmc_handle* hs, int n, int n_burn, const uint64_t* seeds, void* stream) {
    if (!hs || !seeds || n < 1 || n > kMaxBatch || n_burn < 0) return VMC_ERR_INVALID_ARG;
    for (int b = 0; b < n; ++b) {
        if (!hs[b]) return VMC_ERR_INVALID_ARG;
        if (!hs[b]->params_set || !hs[b]->walkers_set) return VMC_ERR_STATE;
        if (hs[b]->wprec != hs[0]->wprec || hs[b]->dev != hs[0]->dev) return VMC_ERR_INVALID_ARG;
        for (int c = 0; c < b; ++c)
            if (hs[c] == hs[b]) return VMC_ERR_INVALID_ARG;
    }
    vmc_ctx* h0 = hs[0];
    cudaStream_t st = (cudaStream_t)stream;
    const bool fp64 = h0->wprec == VMC_FP64;
    std::vector<SampleArgs> args(n);
    std::vector<int> wstart(n + 1, 0);
    size_t wb = 0;
    for (int b = 0; b < n; ++b) {
        sample_args(hs[b], n_burn, seeds[b], args[b]);
        wb = std::max(wb, prep_walkers(hs[b], args[b], fp64));
        wstart[b + 1] = wstart[b] + hs[b]->n_walkers;
    }
    const int wpb = (int)std::min<size_t>(4, h0->smem_optin / wb);
    if (wpb < 1) return VMC_ERR_UNSUPPORTED;
    void* dbuf = nullptr;
    const size_t abytes = round_up(sizeof(SampleArgs) * n, 256);
    int rc = batch_buffer(h0, abytes + sizeof(int) * (n + 1), &dbuf);
    if (rc) return rc;
    SampleArgs* dargs = (SampleArgs*)dbuf;
    int* dws = (int*)((unsigned char*)dbuf + abytes);
    VCK(cudaMemcpyAsync(dargs, args.data(), sizeof(SampleArgs) * n, cudaMemcpyHostToDevice, st));
    VCK(cudaMemcpyAsync(dws, wstart.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
    const size_t smem = wb * wpb;
    const int blocks = (wstart[n] + wpb - 1) / wpb;
    VCK(launch_walkers_batch(fp64, blocks, 32 * wpb, smem, st, dargs, dws, n, wb));
    h0->n_launch++;
    // the host copies of the argument blocks must outlive the launch's copies
    VCK(cudaStreamSynchronize(st));
    int first = VMC_OK;
    for (int b = 0; b < n; ++b) {
        rc = after_sampling(hs[b], st);
        if (rc && !first) first = rc;
    }
    return first;
}

static int measure_device_configs(vmc_ctx* h, int64_t n_s, bool fp64, const double* bw, double* bgrad,
                                  bool to_store, cudaStream_t st) {
    SampleArgs a{};
    a.n_walkers = (int)n_s;
    a.spw = 1;
    a.n_burn = 0;
    a.props_per_sweep = 0;
    a.write_back = 0;
    a.want_energy = bgrad ? 0 : 1;
    a.walker_occ = h->d_mocc;
    a.walker_step = nullptr;
    if (to_store) store_targets(h, a);
    a.bw = bw;
    a.bgrad = bgrad;
    return launch_walkers(h, a, fp64, st);
}

extern "C" int vmc_measure(vmc_handle h, const uint8_t* occ, int64_t n_s, void* stream) {
    if (!h || !occ || n_s < 1 || n_s > h->ncap) return VMC_ERR_INVALID_ARG;
    if (!h->params_set) return VMC_ERR_STATE;
    int rc = check_configs(h, occ, n_s);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    VCK(cudaMemcpyAsync(h->d_mocc, occ, (size_t)n_s * h->N, cudaMemcpyHostToDevice, st));
    rc = measure_device_configs(h, n_s, h->wprec == VMC_FP64, nullptr, nullptr, true, st);
    if (rc) return rc;
    h->n_s = n_s;
    h->obar_ok[0] = h->obar_ok[1] = h->obar_ok[2] = false;
    h->sorted_ok = h->g_ok = h->corr_ok = false;
    rc = transpose_states(h, st);
    if (rc) return rc;
    return read_status(h, st);
}

extern "C" int vmc_sample_stats(vmc_handle h, vmc_sample_stats_t* out, void* stream) {
    if (!h || !out) return VMC_ERR_INVALID_ARG;
    if (h->n_s == 0 || h->spw < 1 || h->n_s != (int64_t)h->n_walkers * h->spw) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = h->n_s;
    if (!h->d_lnps) VCK(h->alloc(&h->d_lnps, h->ncap));
    double* lnps = h->d_lnps;
    int rc = vmc_logpsi(h, lnps, stream);
    if (rc) return rc;
    std::vector<double> lp(n), lr(n), E(n), Ec;
    VCK(cudaMemcpyAsync(lp.data(), lnps, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    VCK(cudaMemcpyAsync(lr.data(), h->d_lnrun, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    VCK(cudaMemcpyAsync(E.data(), h->d_E, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    if (h->refreshed) {
        Ec.resize(n);
        VCK(cudaMemcpyAsync(Ec.data(), h->d_Echain, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    }
    VCK(cudaStreamSynchronize(st));
    vmc_sample_stats_t r{};
    double sd = 0.0, se = 0.0;
    int64_t cnt = 0;
    for (int64_t w = 0; w < h->n_walkers; ++w) {
        const int64_t s0 = w * h->spw;
        for (int j = 1; j < h->spw; ++j) {
            const int64_t s = s0 + j;
            const double d = std::fabs((lr[s] - lr[s0]) - (lp[s] - lp[s0]));
            r.lnpsi_drift_max = std::max(r.lnpsi_drift_max, d);
            sd += d;
            ++cnt;
        }
    }
    r.lnpsi_drift_mean = cnt ? sd / cnt : 0.0;
    r.refreshed = h->refreshed ? 1 : 0;
    if (h->refreshed) {
        for (int64_t s = 0; s < n; ++s) {
            const double d = std::fabs(Ec[s] - E[s]) / std::max(1.0, std::fabs(E[s]));
            r.el_refresh_change_max = std::max(r.el_refresh_change_max, d);
            se += d;
        }
        r.el_refresh_change_mean = se / n;
    }
    *out = r;
    return VMC_OK;
}

extern "C" int vmc_get_samples(vmc_handle h, uint8_t* occ, double* E_L, uint32_t* corr_state, double* pf,
                               int store, void* stream) {
    if (!h) return VMC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    VCK(cudaStreamSynchronize(st));
    const int64_t n = h->n_s;
    if (occ) VCK(cudaMemcpy2D(occ, h->N, h->d_socc, h->Nst, h->N, n, cudaMemcpyDeviceToHost));
    if (E_L) VCK(cudaMemcpy(E_L, h->d_E, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (corr_state && h->ncorr > 0)
        VCK(cudaMemcpy2D(corr_state, sizeof(cstate_t) * h->ncorr, h->d_cidx, sizeof(cstate_t) * h->ncst,
                         sizeof(cstate_t) * h->ncorr, n, cudaMemcpyDeviceToHost));
    if (pf) {
        if (store == VMC_STORE_FP64) {
            if (!h->d_pf64) return VMC_ERR_STATE;
            VCK(cudaMemcpy2D(pf, sizeof(double) * h->P, h->d_pf64, sizeof(double) * h->Pst, sizeof(double) * h->P, n,
                             cudaMemcpyDeviceToHost));
        } else if (store == VMC_STORE_FP32 || store == VMC_STORE_FP32_F32ACC) {
            if (!h->d_pf32) return VMC_ERR_STATE;
            std::vector<float> tmp((size_t)n * h->P);
            VCK(cudaMemcpy2D(tmp.data(), sizeof(float) * h->P, h->d_pf32, sizeof(float) * h->Pst, sizeof(float) * h->P,
                             n, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < tmp.size(); ++i) pf[i] = tmp[i];
        } else if (store == VMC_STORE_BF16) {
            if (!h->d_pf16) return VMC_ERR_STATE;
            std::vector<uint16_t> tmp((size_t)n * h->P);
            VCK(cudaMemcpy2D(tmp.data(), 2 * h->P, h->d_pf16, 2 * h->Pst, 2 * h->P, n, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < tmp.size(); ++i) {
                uint32_t b = (uint32_t)tmp[i] << 16;
                float f;
                memcpy(&f, &b, 4);
                pf[i] = f;
            }
        } else {
            return VMC_ERR_INVALID_ARG;
        }
    }
    return VMC_OK;
}

extern "C" int vmc_logpsi(vmc_handle h, double* out, void* stream) {
    if (!h || !out) return VMC_ERR_INVALID_ARG;
    if (!h->params_set || h->n_s == 0) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    LogPsiArgs a{};
    a.pb = h->pb;
    a.n_s = h->n_s;
    a.s_occ = h->d_socc; a.Nst = h->Nst;
    a.s_cidx = h->d_cidx; a.ncst = h->ncst;
    a.XS = h->N + 1;
    a.warp_bytes = round_up((size_t)h->N * a.XS * 8 + 2 * (size_t)a.XS * 8, 16);
    int wpb = 4;
    size_t smem = a.warp_bytes * wpb;
    a.out = out;
    VCK(cudaFuncSetAttribute(k_logpsi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_logpsi<<<(unsigned)((h->n_s + wpb - 1) / wpb), 32 * wpb, smem, st>>>(a); h->n_launch++;
    VCK(cudaGetLastError());
    return VMC_OK;
}

extern "C" int vmc_logpsi_backward(vmc_handle h, const double* w, double* grad, void* stream) {
    if (!h || (w && !grad)) return VMC_ERR_INVALID_ARG;
    if (!h->params_set || h->n_s == 0) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    VCK(cudaMemcpy2DAsync(h->d_mocc, h->N, h->d_socc, h->Nst, h->N, h->n_s, cudaMemcpyDeviceToDevice, st));
    int rc;
    if (w) {
        VCK(cudaMemsetAsync(grad, 0, sizeof(double) * h->nv, st));
        rc = measure_device_configs(h, h->n_s, true, w, grad, false, st);
    } else {
        rc = measure_device_configs(h, h->n_s, true, nullptr, nullptr, true, st);
        h->obar_ok[0] = h->obar_ok[1] = h->obar_ok[2] = false;
    h->sorted_ok = h->g_ok = h->corr_ok = false;
    }
    if (rc) return rc;
    return read_status(h, st);
}

// ---------------------------------------------------------------------------
// streaming passes over the O store
// ---------------------------------------------------------------------------
template <typename ST, typename AT, int K, bool G>
static int launch_main(vmc_ctx* h, const void* s_pf, const AT* V, const AT* invC, AT* T, const int* stop,
                       cudaStream_t st, int* nblk) {
    const int threads = 512;
    size_t smem = (size_t)h->npf * K * sizeof(AT) * (G ? 2 : 1) + (size_t)h->M * 4 + 16 * 64;
    if (smem > h->smem_optin) { set_err("pairing block does not fit in shared memory"); return VMC_ERR_UNSUPPORTED; }
    auto kern = k_sr_main<ST, AT, K, G>;
    VCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    VCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    per_sm = std::max(1, std::min(per_sm, 4));
    int grid = h->nsm * per_sm;
    int64_t need = (h->n_s + 15) / 16;
    if (need < grid) grid = (int)std::max<int64_t>(1, need);
    if ((size_t)grid * h->npf * K * sizeof(AT) > h->pfpart_bytes) return VMC_ERR_UNSUPPORTED;
    const int kind = sizeof(ST) == 8 ? VMC_STORE_FP64
                     : sizeof(ST) == 2 ? VMC_STORE_BF16
                     : (sizeof(AT) == 8 ? VMC_STORE_FP32 : VMC_STORE_FP32_F32ACC);
    vmc_ctx::PassRec rec{};
    if (h->prof) {
        rec.a = h->get_event();
        rec.b = h->get_event();
        rec.kind = kind;
        rec.bytes = (double)h->n_s * (2.0 * h->ncorr + h->N + (double)h->P * sizeof(ST));
        VCK(cudaEventRecord(rec.a, st));
    }
    MainArgs<AT> a{};
    a.pb = h->pb;
    a.n_s = h->n_s;
    a.s_occ = h->d_socc; a.Nst = h->Nst;
    a.s_cidx = h->d_cidx; a.ncst = h->ncst;
    a.s_pf = s_pf; a.Pst = h->Pst;
    a.V = V; a.invC = invC; a.T = T;
    a.pf_partial = (AT*)h->d_pfpart;
    a.stop = stop;
    kern<<<grid, threads, smem, st>>>(a);
    VCK(cudaGetLastError());
    h->n_launch++;
    if (h->prof) {
        VCK(cudaEventRecord(rec.b, st));
        h->recs.push_back(rec);
    }
    *nblk = grid;
    return VMC_OK;
}

// TMA-staged pass for FP32 accumulation (BF16 / FP32 stores); returns
// VMC_ERR_UNSUPPORTED when the problem does not fit its layout, and the
// caller then uses the generic pass.
template <typename ST, int K>
static int launch_stream(vmc_ctx* h, const void* s_pf, const float* V, const float* invC, float* T, const int* stop,
                         cudaStream_t st, int* nblk) {
    if (h->nu > 32 || h->nd > 32) return VMC_ERR_UNSUPPORTED;
    const size_t buf = (size_t)round_up(h->Nst + h->Pst * (int64_t)sizeof(ST), 128);
    const size_t tabs = (size_t)((h->nu >> 1) + (h->nd >> 1)) * 32 * 4;
    const size_t fixed =
        (size_t)round_up((int64_t)h->npf * K * 8 + (int64_t)(h->ncorr + 1) * 4 + (int64_t)tabs, 16) + 128;
    // BF16 with one vector: register-cached variant (16 warps, 128 registers)
    const bool cached = sizeof(ST) == 2 && K == 1 && h->stream_cached;
    int nw = cached ? 16 : 24;
    while (nw > 1 && fixed + (size_t)nw * (2 * buf + 16) > h->smem_optin) --nw;
    const size_t smem = fixed + (size_t)nw * (2 * buf + 16);
    if (smem > h->smem_optin || nw < 4) return VMC_ERR_UNSUPPORTED;
    auto kern = cached ? k_sr_stream_bf16c : k_sr_stream<ST, K>;
    VCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = h->nsm;
    int64_t need = (h->n_s + nw - 1) / nw;
    if (need < grid) grid = (int)std::max<int64_t>(1, need);
    if ((size_t)grid * h->npf * K * sizeof(float) > h->pfpart_bytes) return VMC_ERR_UNSUPPORTED;
    const int kind = sizeof(ST) == 2 ? VMC_STORE_BF16 : VMC_STORE_FP32_F32ACC;
    vmc_ctx::PassRec rec{};
    if (h->prof) {
        rec.a = h->get_event();
        rec.b = h->get_event();
        rec.kind = kind;
        rec.bytes = (double)h->n_s * (2.0 * h->ncorr + h->N + (double)h->P * sizeof(ST));
        VCK(cudaEventRecord(rec.a, st));
    }
    StreamArgs a{};
    a.pb = h->pb;
    a.n_s = h->n_s;
    a.s_occ = h->d_socc; a.Nst = h->Nst;
    a.s_cidx = h->d_cidx; a.ncst = h->ncst;
    a.s_pf = s_pf; a.Pst = h->Pst; a.st_bytes = (int)sizeof(ST);
    a.V = V; a.invC = invC; a.T = T;
    a.pf_partial = (float*)h->d_pfpart;
    a.stop = stop;
    a.status = h->d_status;
    a.spin_limit = h->wait_limit;
    a.buf_bytes = buf;
    kern<<<grid, 32 * nw, smem, st>>>(a);
    VCK(cudaGetLastError());
    h->n_launch++;
    if (h->prof) {
        VCK(cudaEventRecord(rec.b, st));
        h->recs.push_back(rec);
    }
    *nblk = grid;
    return VMC_OK;
}

// correlator scatter: one thread-block cluster of kCorrCluster CTAs per
// correlator, the sums over samples go to d_corrraw
template <typename AT, int K>
static int launch_corr(vmc_ctx* h, const AT* T, const int* stop, cudaStream_t st) {
    if (h->ncorr == 0) return VMC_OK;
    size_t smem = (size_t)h->maxd * K * sizeof(AT);
    CorrArgs<AT> a{};
    a.pb = h->pb;
    a.n_s = h->n_s;
    a.cidxT = h->d_cidxT;
    a.T = T;
    a.corr_raw = (AT*)h->d_corrraw;
    a.units = h->d_units;
    a.stop = stop;
    VCK(cudaMemsetAsync(h->d_corrraw, 0, sizeof(AT) * h->ncp * K, st));
    if (smem + 1024 > h->smem_optin) {   // histograms beyond shared memory: global additions
        const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((h->n_s + 255) / 256, 64)),
                        (unsigned)h->ncorr);
        k_corr_scatter_global<AT, K><<<grid, 256, 0, st>>>(a); h->n_launch++;
        VCK(cudaGetLastError());
        return VMC_OK;
    }
    auto kern = k_corr_scatter<AT, K>;
    VCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<h->n_units * kCorrCluster, 256, smem, st>>>(a); h->n_launch++;
    VCK(cudaGetLastError());
    return VMC_OK;
}

template <typename AT>
static int reduce_pf(vmc_ctx* h, int nblk, int K, cudaStream_t st) {
    const int n = h->npf * K;
    k_reduce_pf<AT><<<(n + 31) / 32, 256, 0, st>>>((const AT*)h->d_pfpart, nblk, n, (AT*)h->d_pfraw); h->n_launch++;
    VCK(cudaGetLastError());
    return VMC_OK;
}

// blocks of the unrolled vector kernels (4 elements per thread); their K
// partial dots per block go to one slot of kNumPart * kMaxK doubles
static int vgrid(const vmc_ctx* h, int K = 1) {
    int64_t g = (h->nv + 1023) / 1024;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)kNumPart * kMaxK / K));
}

// blocks of the gradient finalize kernel
static int fin_grid(const vmc_ctx* h, int K = 1) {
    int64_t g = (h->nv + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)kNumPart * kMaxK / K));
}

static int ensure_corr_runs(vmc_ctx* h, cudaStream_t st);

// Build G (sample-major packed) and T (parameter-major, per 65,536-sample
// chunk) from the BF16 store, once per set of samples.
static int ensure_G(vmc_ctx* h, cudaStream_t st) {
    if (h->g_ok) return VMC_OK;
    if (!h->d_G || h->n_s == 0) return VMC_ERR_STATE;
    k_build_G<<<(unsigned)((h->n_s + 7) / 8), 256, 0, st>>>(h->pb, h->n_s, h->d_socc, h->Nst, h->d_pf16, h->Pst,
                                                           h->d_fulltab, h->gwq, h->Gst, h->d_G, h->d_G16,
                                                           h->Gst16); h->n_launch++;
    VCK(cudaGetLastError());
    h->g_ok = true;
    return VMC_OK;
}

static int ensure_sorted(vmc_ctx* h, cudaStream_t st) {
    if (h->sorted_ok) return VMC_OK;
    if (!h->d_G || h->n_s == 0) return VMC_ERR_STATE;
    int rc0 = ensure_G(h, st);
    if (rc0) return rc0;
    const size_t smem = (size_t)h->npf * 4;
    VCK(cudaFuncSetAttribute(k_count_G, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    VCK(cudaFuncSetAttribute(k_fill_T, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * smem)));
    const int nchunk = (int)((h->n_s + kTChunk - 1) / kTChunk);
    // run padding must read as weight 0
    VCK(cudaMemsetAsync(h->d_Tsort, 0, sizeof(uint32_t) * h->t_chunk * nchunk, st));
    for (int c = 0; c < nchunk; ++c) {
        const int64_t sb = (int64_t)c * kTChunk, se = std::min<int64_t>(h->n_s, sb + kTChunk);
        uint32_t* base = h->d_base + (size_t)c * (h->npf + 1);
        k_count_G<<<h->sort_nblk, 512, smem, st>>>(h->d_G, h->Gst, h->P, sb, se, h->npf, h->d_counts); h->n_launch++;
        k_scan_blocks<<<(h->npf + 255) / 256, 256, 0, st>>>(h->d_counts, h->sort_nblk, h->npf, h->d_total); h->n_launch++;
        k_scan_params<<<1, 1024, 0, st>>>(h->d_total, h->npf, (uint32_t)(c * h->t_chunk), base); h->n_launch++;
        k_fill_T<<<h->sort_nblk, 512, 2 * smem, st>>>(h->d_G, h->Gst, h->P, sb, se, h->npf, h->d_counts, base,
                                                  h->d_Tsort); h->n_launch++;
        VCK(cudaGetLastError());
    }
    if (h->rank_T) {
        k_rank_T<<<h->nsm * 8, 256, 0, st>>>(h->d_Tsort, (int64_t)h->t_chunk, nchunk, h->d_base, h->npf, h->n_s);
        h->n_launch++;
        VCK(cudaGetLastError());
    }
    int rc = ensure_corr_runs(h, st);
    if (rc) return rc;
    h->sorted_ok = true;
    return VMC_OK;
}

// Correlator runs (the samples of every correlator parameter grouped by
// parameter) and the work items of their scatter, once per set of samples.
static int ensure_corr_runs(vmc_ctx* h, cudaStream_t st) {
    if (h->corr_ok) return VMC_OK;
    if (!h->d_Tc || h->n_s == 0) return VMC_ERR_STATE;
    if (h->ncorr > 0) {
        // (class, slice) grid: a class shared by many correlators spreads over
        // several CTAs
        const bool shist = (size_t)h->maxd * 4 + 1024 <= h->smem_optin;   // shared-memory counters fit
        const size_t csm = shist ? (size_t)h->maxd * 4 : 0;
        const int nsl = std::max(1, std::min(64, (2 * h->nsm + h->n_class - 1) / h->n_class));
        const dim3 cgrid((unsigned)h->n_class, (unsigned)nsl);
        VCK(cudaFuncSetAttribute(k_count_C, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm));
        VCK(cudaMemsetAsync(h->d_ccount, 0, sizeof(uint32_t) * h->ncp, st));
        k_count_C<<<cgrid, 512, csm, st>>>(h->pb, h->n_s, h->d_cidxT, h->d_ccount, shist ? 1 : 0); h->n_launch++;
        k_scan_params<<<1, 1024, 0, st>>>(h->d_ccount, (int)h->ncp, 0u, h->d_cbase); h->n_launch++;
        VCK(cudaMemcpyAsync(h->d_ccount, h->d_cbase, sizeof(uint32_t) * h->ncp, cudaMemcpyDeviceToDevice, st));
        k_fill_C<<<cgrid, 512, 0, st>>>(h->pb, h->n_s, h->d_cidxT, h->d_ccount, h->d_Tc); h->n_launch++;
        // work items of the correlator scatter
        const int64_t ng = (h->ncp + 31) / 32;
        k_corr_item_count<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(h->d_cbase, h->ncp, h->d_nitems); h->n_launch++;
        k_scan_params<<<1, 1024, 0, st>>>(h->d_nitems, (int)ng, 0u, h->d_item_base); h->n_launch++;
        k_corr_item_fill<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(h->d_cbase, h->ncp, h->d_item_base,
                                                                        h->d_items); h->n_launch++;
        VCK(cudaGetLastError());
    }
    h->corr_ok = true;
    return VMC_OK;
}

// gather kernel holding a whole G row in registers: U 16-byte loads per lane
using GatherKern = void (*)(SortedArgs);
template <int K>
static GatherKern gather_kernel(int u) {
    if constexpr (K == 1) {
        static const GatherKern tab[16] = {
            k_gather_G<1, 1>,  k_gather_G<1, 2>,  k_gather_G<1, 3>,  k_gather_G<1, 4>,
            k_gather_G<1, 5>,  k_gather_G<1, 6>,  k_gather_G<1, 7>,  k_gather_G<1, 8>,
            k_gather_G<1, 9>,  k_gather_G<1, 10>, k_gather_G<1, 11>, k_gather_G<1, 12>,
            k_gather_G<1, 13>, k_gather_G<1, 14>, k_gather_G<1, 15>, k_gather_G<1, 16>};
        return u >= 1 && u <= 16 ? tab[u - 1] : nullptr;
    } else {
        if (u <= 4) return k_gather_G<K, 4>;
        if (u <= 8) return k_gather_G<K, 8>;
        if (u <= 13) return k_gather_G<K, 13>;   // 56 electrons: 1,540 elements in 13 words per lane
        if (u <= 16) return k_gather_G<K, 16>;
        return nullptr;
    }
}

// the sorted product applies: BF16 store with its sorted copies, the gather's
// table within shared memory, at most 128 correlators, rows of at most 2048
// elements
template <int K>
static bool sorted_usable(const vmc_ctx* h) {
    if (!h->use_sorted || !h->d_G || h->ncorr > 32 * kCorrPerLane) return false;
    if ((size_t)h->npf * K * 4 + (size_t)(h->ncorr + 1) * 4 > h->smem_optin) return false;   // gather table
    // scatter: the chunk's t_s, the group's run ends and the correlator slots
    if ((size_t)kTChunk * K * 4 + (size_t)(kScatterMaxPQ + 1) * 4 + (size_t)scatter_threads(K) * 4 * K + 1024 >
        h->smem_optin)
        return false;
    return gather_kernel<K>((int)((h->Gst / 4 + 31) / 32)) != nullptr;
}

// correlator half of the single pass's finish as shared-memory histograms
// when every class's 4^m amplitudes (K values each) fit 64 KB: (class, slice)
// CTAs with about two CTAs per SM in total; else the correlator work items
static size_t corr_hist_setup(const vmc_ctx* h, int K, SortedArgs* a) {
    a->cidxT = h->d_cidxT;
    a->nhist = 0;
    a->hist_slices = 1;
    if (h->ncorr == 0) { a->ncb = 0; return 0; }
    const size_t bytes = (size_t)h->maxd * K * sizeof(float);
    if (bytes > 65536) { a->ncb = (int)((h->max_items + 7) / 8); return 0; }
    const int64_t by_n = std::max<int64_t>(1, h->n_s / 1024);
    const int nsl = (int)std::max<int64_t>(1, std::min<int64_t>(by_n, (2 * h->nsm + h->n_class - 1) / h->n_class));
    a->hist_slices = nsl;
    a->nhist = h->n_class * nsl;
    a->ncb = 0;
    return bytes;
}

// product path of a K-vector product (VMC_PATH_*): the caller's choice, or
// under AUTO the autotuner's (default: the sorted two-pass product)
static int product_path(const vmc_ctx* h, int K) {
    if (h->path != VMC_PATH_AUTO) return h->path;
    return K == 1 ? h->auto_path : h->auto_path4;
}

// the compact gather applies: its copy exists, at most 128 correlators, the
// v table, the word table and one occupation row per warp in shared memory,
// rows of at most 8 words per lane
static size_t compact_smem(const vmc_ctx* h) {
    const size_t nw16 = (size_t)(h->Gst16 / 8);
    return (size_t)h->npf * 4 + (size_t)(h->ncorr + 1) * 4 + (nw16 + 7) / 8 * 16 +
           (size_t)(kCompactThreads / 32) * (h->Nst + 16);
}
static bool compact_usable(const vmc_ctx* h) {
    if (!h->use_compact || !h->d_G16 || !h->d_wtab || h->ncorr > 32 * kCorrPerLane) return false;
    if (compact_smem(h) + 1024 > h->smem_optin) return false;
    const int64_t u = (h->Gst16 / 8 + 31) / 32;
    return u >= 1 && u <= 8;
}

using CompactKern = void (*)(SortedArgs, const uint16_t*, int64_t, const uint16_t*, const uint8_t*, int);
static CompactKern compact_kernel(int64_t u) {
    static const CompactKern tab[5] = {k_gather_C<4>, k_gather_C<5>, k_gather_C<6>, k_gather_C<7>, k_gather_C<8>};
    return tab[std::max<int64_t>(0, u - 4)];
}

// Launch shapes of the sorted product for K vectors.  Gather: as many CTAs
// as fit on the GPU, at most one per warp-row of samples.  Scatter: one wave
// of pairing CTAs over the chunks, each CTA a group of consecutive
// parameters of one chunk (at least one per warp).  The correlator half:
// histograms of the chunk's t_s inside the pairing CTAs when they fit beside
// the chunk table (K >= scatter_in_cta_mink), else (class, sample slice)
// histogram CTAs ahead of the pairing CTAs, else the correlator work items
// (CTAs of their own ahead, or after each pairing CTA's runs).
template <int K>
static int plan_sorted(vmc_ctx* h, bool compact, SortedArgs a, vmc_ctx::SortedLaunch* L) {
    const int sthreads = scatter_threads(K), swarps = sthreads / 32;
    {
        const int gthreads = compact ? kCompactThreads : gather_threads(K), gwarps = gthreads / 32;
        const size_t smem = compact ? compact_smem(h) : (size_t)h->npf * K * 4 + (size_t)(h->ncorr + 1) * 4;
        const void* gk = compact ? (const void*)compact_kernel((h->Gst16 / 8 + 31) / 32)
                                 : (const void*)gather_kernel<K>((int)((h->Gst / 4 + 31) / 32));
        VCK(cudaFuncSetAttribute(gk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        VCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gk, gthreads, smem));
        int grid = h->nsm * std::max(1, per_sm);
        const int64_t need = (h->n_s + gwarps - 1) / gwarps;
        if (need < grid) grid = (int)std::max<int64_t>(1, need);
        L->ggrid = std::min(grid, kNumPart * kMaxK);   // one partial slot of tt sums
        L->gsmem = smem;
    }
    const size_t ssm_tab = (size_t)kTChunk * K * sizeof(float);
    const int pq_cap = std::min(std::max(h->npf, swarps), kScatterMaxPQ);
    const size_t run_bytes = ((size_t)(pq_cap + 1) * 4 + 15) / 16 * 16;
    const size_t static_bytes = (size_t)sthreads * K * sizeof(float) + 1024;
    size_t hsm = 0;
    a.nhist = 0;
    a.hist_slices = 1;
    a.ncb = 0;
    a.corr_in_cta = 0;
    a.hist_cap = 0;
    if (h->ncorr > 0) {
        const int64_t one = (int64_t)h->maxd * K;
        const int cap = (int)std::max<int64_t>(one, std::min<int64_t>(one * swarps, 8192));
        if (K >= h->scatter_in_cta_mink && ssm_tab + run_bytes + (size_t)cap * 4 + static_bytes <= h->smem_optin) {
            a.corr_in_cta = 1;
            a.hist_cap = cap;
        } else if (h->scatter_corr_hist && (hsm = corr_hist_setup(h, K, &a)) > 0) {
            a.ncb = 0;
        } else {
            hsm = 0;
            a.nhist = 0;
            a.hist_slices = 1;
            a.ncb = h->scatter_corr_front ? (int)((h->max_items + swarps - 1) / swarps) : 0;
        }
    }
    // shared memory for a group of pq run ends: one estimate for the
    // occupancy query, then the group size it gives
    const size_t in_cta = (size_t)a.hist_cap * 4;
    auto run_of = [](int pq) { return ((size_t)(pq + 1) * 4 + 15) / 16 * 16; };
    auto smem_of = [&](int pq) { return std::max(hsm, ssm_tab + run_of(pq) + in_cta); };
    const int pq_est = std::min(pq_cap, std::max(swarps, h->npf / h->nsm + 64));
    VCK(cudaFuncSetAttribute(k_scatter_T<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_of(pq_cap)));
    int per = 0;
    VCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_scatter_T<K>, sthreads, smem_of(pq_est)));
    const int64_t resident = (int64_t)h->nsm * std::max(1, per);
    const int64_t target = resident * (K == 1 ? h->scatter_waves1 : h->scatter_waves4);
    int ngrp = (int)std::max<int64_t>(1, std::min<int64_t>(h->npf, (target + a.nchunk - 1) / a.nchunk));
    L->pq_per_cta = std::min(pq_cap, std::max(swarps, (h->npf + ngrp - 1) / ngrp));
    ngrp = (h->npf + L->pq_per_cta - 1) / L->pq_per_cta;
    L->hist_off = (int)(ssm_tab + run_of(L->pq_per_cta));   // bytes: the in-CTA histograms
    L->nhist = a.nhist; L->hist_slices = a.hist_slices; L->ncb = a.ncb;
    L->corr_in_cta = a.corr_in_cta; L->hist_cap = a.hist_cap;
    L->sgrid = a.nhist + a.ncb + a.nchunk * ngrp;
    L->ssm = smem_of(L->pq_per_cta);
    L->n_s = h->n_s;
    L->compact = compact;
    return VMC_OK;
}

// gather + parameter-major scatter for the BF16 store; the centered t_s go to
// Tv, the pairing sums to d_pfraw and the correlator sums to d_corrraw (FP32)
template <int K>
static int launch_sorted(vmc_ctx* h, const float* V, const float* invC, const double* obv_part, float* Tv,
                         const int* stop, cudaStream_t st, double* tt_part = nullptr, bool craw_zero = false) {
    if (!sorted_usable<K>(h)) return VMC_ERR_UNSUPPORTED;
    int rc = ensure_sorted(h, st);
    if (rc) return rc;
    vmc_ctx::PassRec rec{};
    if (h->prof) {
        rec.a = h->get_event();
        rec.b = h->get_event();
        rec.kind = VMC_STORE_BF16;
        rec.bytes = (double)h->n_s * (2.0 * h->ncorr + h->N + (double)h->P * 2);
        VCK(cudaEventRecord(rec.a, st));
    }
    SortedArgs a{};
    a.pb = h->pb;
    a.n_s = h->n_s;
    a.s_cidx = h->d_cidx; a.ncst = h->ncst;
    a.G = h->d_G; a.Pst = h->Gst;
    a.V = V; a.invC = invC; a.Tv = Tv;
    a.obv_part = obv_part; a.n_obv_part = vgrid(h, K);
    a.T = h->d_Tsort; a.base = h->d_base; a.nchunk = (int)((h->n_s + kTChunk - 1) / kTChunk);
    a.part = h->d_tpart; a.done = h->d_tdone;
    a.raw = (float*)h->d_pfraw;
    a.Tc = h->d_Tc; a.cbase = h->d_cbase; a.craw = (float*)h->d_corrraw;
    a.items = h->d_items;
    a.n_items = h->d_item_base + (h->ncp + 31) / 32;
    a.tt_part = tt_part;
    a.stop = stop;
    const bool compact = K == 1 && product_path(h, 1) == VMC_PATH_COMPACT && compact_usable(h);
    // the launch shapes depend on the problem, K, the gather kind and n_s
    // only: worked out (attributes, occupancy queries) once and kept, so the
    // inner CG iteration issues its launches without host-side queries
    vmc_ctx::SortedLaunch& L = h->sorted_launch[K == 1 ? 0 : K == 2 ? 1 : 2];
    if (L.n_s != h->n_s || L.compact != compact) {
        int rc2 = plan_sorted<K>(h, compact, a, &L);
        if (rc2) return rc2;
    }
    a.nhist = L.nhist; a.hist_slices = L.hist_slices; a.ncb = L.ncb;
    a.corr_in_cta = L.corr_in_cta; a.hist_cap = L.hist_cap; a.hist_off = L.hist_off; a.pq_per_cta = L.pq_per_cta;
    a.cidxT = h->d_cidxT;
    if (compact) {
        // the compact gather over G16 (occupation rows give the indices)
        compact_kernel((h->Gst16 / 8 + 31) / 32)<<<L.ggrid, kCompactThreads, L.gsmem, st>>>(
            a, h->d_G16, h->Gst16, h->d_wtab, h->d_socc, h->Nst);
    } else {
        gather_kernel<K>((int)((h->Gst / 4 + 31) / 32))<<<L.ggrid, gather_threads(K), L.gsmem, st>>>(a);
    }
    h->n_launch++;
    h->last_gather_grid = L.ggrid;
    // correlator sums accumulate into zero (the fused CG update re-zeroes
    // them as it reads them, so its products skip this)
    if (h->ncp > 0 && !craw_zero) VCK(cudaMemsetAsync(h->d_corrraw, 0, sizeof(float) * h->ncp * K, st));
    k_scatter_T<K><<<L.sgrid, scatter_threads(K), L.ssm, st>>>(a);
    h->n_launch++;
    VCK(cudaGetLastError());
    if (h->prof) {
        VCK(cudaEventRecord(rec.b, st));
        h->recs.push_back(rec);
    }
    return VMC_OK;
}

// Fused single-pass product over G (fused.cu): the BF16 store's sorted rows,
// one vector; six private pairing images and the v table in shared memory.
static size_t fused_smem(const vmc_ctx* h) {
    return (size_t)h->npf * 4 * (1 + kFusedImages) + (size_t)(h->ncorr + 1) * 4;
}

static bool fused_usable(const vmc_ctx* h) {
    if (!h->use_fused || !h->d_G || h->ncorr > 32 * kCorrPerLane) return false;
    if ((size_t)h->nsm * h->npf * sizeof(float) > h->pfpart_bytes) return false;
    if (fused_smem(h) + 512 > h->smem_optin) return false;
    return (h->gwq + 31) / 32 <= 4;
}

using FusedKern = void (*)(SortedArgs, float*, int);
static FusedKern fused_kernel(int u) {
    static const FusedKern tab[4] = {k_sv_fused<1>, k_sv_fused<2>, k_sv_fused<3>, k_sv_fused<4>};
    return u >= 1 && u <= 4 ? tab[u - 1] : nullptr;
}

// one pass over G: centered t_s to Tv, the pairing sums to d_pfraw and the
// correlator sums to d_corrraw (FP32), as launch_sorted
static int launch_fused(vmc_ctx* h, const float* V, const float* invC, const double* obv_part, float* Tv,
                        const int* stop, cudaStream_t st, double* tt_part = nullptr, bool craw_zero = false) {
    if (!fused_usable(h)) return VMC_ERR_UNSUPPORTED;
    int rc = ensure_G(h, st);
    if (!rc) rc = ensure_corr_runs(h, st);
    if (rc) return rc;
    vmc_ctx::PassRec rec{};
    if (h->prof) {
        rec.a = h->get_event();
        rec.b = h->get_event();
        rec.kind = VMC_STORE_BF16;
        rec.bytes = (double)h->n_s * (2.0 * h->ncorr + h->N + (double)h->P * 2);
        VCK(cudaEventRecord(rec.a, st));
    }
    SortedArgs a{};
    a.pb = h->pb;
    a.n_s = h->n_s;
    a.s_cidx = h->d_cidx; a.ncst = h->ncst;
    a.G = h->d_G; a.Pst = h->Gst;
    a.V = V; a.invC = invC; a.Tv = Tv;
    a.obv_part = obv_part; a.n_obv_part = vgrid(h, 1);
    a.raw = (float*)h->d_pfraw;
    a.Tc = h->d_Tc; a.cbase = h->d_cbase; a.craw = (float*)h->d_corrraw;
    a.items = h->d_items;
    a.n_items = h->d_item_base + (h->ncp + 31) / 32;
    const size_t hsm = corr_hist_setup(h, 1, &a);
    a.tt_part = tt_part;
    a.stop = stop;
    const size_t smem = fused_smem(h);
    auto fk = fused_kernel((h->gwq + 31) / 32);
    VCK(cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t need = (h->n_s + kFusedImages - 1) / kFusedImages;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(h->nsm, need));
    fk<<<grid, kFusedWarps * 32, smem, st>>>(a, (float*)h->d_pfpart, h->gwq); h->n_launch++;
    VCK(cudaGetLastError());
    h->last_fused_grid = grid;
    if (h->ncp > 0 && !craw_zero) VCK(cudaMemsetAsync(h->d_corrraw, 0, sizeof(float) * h->ncp, st));
    if (hsm) VCK(cudaFuncSetAttribute(k_sv_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm));
    k_sv_finish<<<a.nhist + a.ncb + (h->npf + 255) / 256, 256, hsm, st>>>(a, (const float*)h->d_pfpart, grid);
    h->n_launch++;
    VCK(cudaGetLastError());
    if (h->prof) {
        VCK(cudaEventRecord(rec.b, st));
        h->recs.push_back(rec);
    }
    return VMC_OK;
}

// out = (S + shift I) V with K vectors, V/out in AT precision ([K][nv]), over
// store s_pf whose sample means are Obar of kind `kind`.  obv_part holds
// vgrid(h, K) partial dots Obar . V unless null (then computed first: the
// sorted pass centers t_s with it); dot_part receives vgrid(h, K) partial
// dots out . V.
template <typename ST, typename AT, int K>
static int apply_S_impl(vmc_ctx* h, const void* s_pf, int kind, const AT* V, AT* out, double shift,
                        const int* stop, const double* obv_part, double* dot_part, cudaStream_t st) {
    const AT* invC;
    if (sizeof(AT) == 8) invC = (const AT*)h->d_invC64;
    else invC = (const AT*)h->d_invC32;
    const double* Obar = h->d_Obar[kind];
    const AT* ObarA = sizeof(AT) == 8 ? (const AT*)h->d_Obar[kind] : (const AT*)h->d_Obar32[kind];
    AT* T = (AT*)h->d_T;
    if (!obv_part) {
        k_dot_part<double, AT, K><<<vgrid(h, K), 256, 0, st>>>(Obar, V, h->nv, h->part(0), stop); h->n_launch++;
        VCK(cudaGetLastError());
        obv_part = h->part(0);
    }
    int nblk = 0;
    int rc = VMC_ERR_UNSUPPORTED;
    bool sorted = false;
    const int path = product_path(h, K);
    if constexpr (sizeof(AT) == 4 && sizeof(ST) == 2 && K == 1) {
        if (path == VMC_PATH_FUSED) {
            rc = launch_fused(h, (const float*)V, (const float*)invC, obv_part, (float*)T, stop, st);
            if (rc != VMC_OK && rc != VMC_ERR_UNSUPPORTED) return rc;
            sorted = rc == VMC_OK;
        }
    }
    if constexpr (sizeof(AT) == 4 && sizeof(ST) == 2) {
        if (!sorted && (path == VMC_PATH_SORTED || path == VMC_PATH_FUSED || path == VMC_PATH_COMPACT) &&
            h->use_sorted && h->d_G) {
            rc = launch_sorted<K>(h, (const float*)V, (const float*)invC, obv_part, (float*)T, stop, st);
            if (rc != VMC_OK && rc != VMC_ERR_UNSUPPORTED) return rc;
            sorted = rc == VMC_OK;
        }
    }
    if constexpr (sizeof(AT) == 4 && K <= 2) {
        if (rc == VMC_ERR_UNSUPPORTED && path != VMC_PATH_GENERIC && h->use_stream)
            rc = launch_stream<ST, K>(h, s_pf, (const float*)V, (const float*)invC, (float*)T, stop, st, &nblk);
    }
    if (rc == VMC_ERR_UNSUPPORTED) rc = launch_main<ST, AT, K, true>(h, s_pf, V, invC, T, stop, st, &nblk);
    if (rc) return rc;
    if (!sorted) {   // the sorted pass scatters the correlators itself
        rc = launch_corr<AT, K>(h, T, stop, st);
        if (rc) return rc;
        rc = reduce_pf<AT>(h, nblk, K, st);
        if (rc) return rc;
    }
    FinArgs<AT, AT> f{};
    f.pb = h->pb;
    f.n_s = h->n_s;
    f.inv_n = 1.0 / (double)h->n_s;
    f.centered = sorted ? 1 : 0;
    f.pf_partial = (const AT*)h->d_pfpart;
    f.pf_raw = (const AT*)h->d_pfraw;
    f.corr_raw = (const AT*)h->d_corrraw;
    f.invC = invC;
    f.ObarA = ObarA;
    f.obv_part = obv_part;
    f.n_obv_part = vgrid(h, K);
    f.V = V;
    f.shift = shift;
    f.out = out;
    f.dot_part = dot_part;
    f.stop = stop;
    k_finalize_S<AT, AT, K><<<vgrid(h, K), 256, 0, st>>>(f); h->n_launch++;
    VCK(cudaGetLastError());
    return VMC_OK;
}

static int store_kind(int store) {
    switch (store) {
        case VMC_STORE_FP64: return 0;
        case VMC_STORE_FP32:
        case VMC_STORE_FP32_F32ACC: return 1;
        case VMC_STORE_BF16: return 2;
        default: return -1;
    }
}

static const void* store_ptr(const vmc_ctx* h, int kind) {
    return kind == 0 ? (const void*)h->d_pf64 : kind == 1 ? (const void*)h->d_pf32 : (const void*)h->d_pf16;
}

// Obar_kind = mean of O over the samples as stored in store `kind`, and
// g = <E_L O> - <E_L> Obar (both FP64 accumulation): one pass with t_s = (1, E_s).
static int gradient_pass(vmc_ctx* h, int kind, double* g, cudaStream_t st) {
    const void* src = store_ptr(h, kind);
    if (!src) return VMC_ERR_STATE;
    double* T = (double*)h->d_T;
    k_build_T_grad<<<kNumPart, 256, 0, st>>>(h->d_E, h->n_s, T, h->part(1)); h->n_launch++;
    VCK(cudaGetLastError());
    int nblk = 0, rc;
    if (kind == 0) rc = launch_main<double, double, 2, false>(h, src, nullptr, nullptr, T, nullptr, st, &nblk);
    else if (kind == 1) rc = launch_main<float, double, 2, false>(h, src, nullptr, nullptr, T, nullptr, st, &nblk);
    else rc = launch_main<__nv_bfloat16, double, 2, false>(h, src, nullptr, nullptr, T, nullptr, st, &nblk);
    if (rc) return rc;
    rc = launch_corr<double, 2>(h, T, nullptr, st);
    if (rc) return rc;
    rc = reduce_pf<double>(h, nblk, 2, st);
    if (rc) return rc;
    FinArgs<double, double> f{};
    f.pb = h->pb;
    f.n_s = h->n_s;
    f.inv_n = 1.0 / (double)h->n_s;
    f.pf_partial = (const double*)h->d_pfpart;
    f.pf_raw = h->d_pfraw;
    f.corr_raw = h->d_corrraw;
    f.invC = h->d_invC64;
    f.Obar_out = h->d_Obar[kind];
    f.g_out = g;
    f.E_sum = h->part(1);
    f.n_E_part = kNumPart;
    k_finalize_grad<double><<<fin_grid(h), 256, 0, st>>>(f); h->n_launch++;
    k_cast<float><<<kNumPart, 256, 0, st>>>(h->d_Obar[kind], h->d_Obar32[kind], h->nv, 1.0); h->n_launch++;
    VCK(cudaGetLastError());
    h->obar_ok[kind] = true;
    return VMC_OK;
}

// the covariance of a store is formed with the mean of that same store, so
// every low-precision operator is itself a covariance (positive semidefinite)
static int ensure_obar(vmc_ctx* h, int kind, cudaStream_t st) {
    if (h->obar_ok[kind]) return VMC_OK;
    return gradient_pass(h, kind, h->d_t64, st);
}

extern "C" int sr_gradient(vmc_handle h, double* g, double* e_stats, int store, void* stream) {
    if (!h || !g) return VMC_ERR_INVALID_ARG;
    if (h->n_s == 0) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    if (store != VMC_STORE_FP64 && store != VMC_STORE_FP32 && store != VMC_STORE_BF16) return VMC_ERR_INVALID_ARG;
    int rc = gradient_pass(h, store_kind(store), g, st);
    if (rc) return rc;
    if (e_stats) {
        std::vector<double> E(h->n_s);
        VCK(cudaMemcpyAsync(E.data(), h->d_E, sizeof(double) * h->n_s, cudaMemcpyDeviceToHost, st));
        VCK(cudaStreamSynchronize(st));
        double m = 0.0;
        for (double e : E) m += e;
        m /= (double)h->n_s;
        double v = 0.0;
        for (double e : E) v += (e - m) * (e - m);
        v /= (double)h->n_s;
        // standard error from per-walker means (blocking over walkers)
        int64_t nw = h->n_s / h->spw;
        double se = 0.0;
        if (nw > 1 && h->n_s == (int64_t)h->n_walkers * h->spw) {
            double sm = 0.0, ss = 0.0;
            for (int64_t w = 0; w < nw; ++w) {
                double a = 0.0;
                for (int j = 0; j < h->spw; ++j) a += E[w * h->spw + j];
                a /= h->spw;
                sm += a;
                ss += a * a;
            }
            sm /= nw;
            double var_w = (ss / nw - sm * sm) * nw / (nw - 1);
            se = std::sqrt(std::max(0.0, var_w) / nw);
        } else {
            se = std::sqrt(v / std::max<int64_t>(1, h->n_s - 1));
        }
        e_stats[0] = m;
        e_stats[1] = v;
        e_stats[2] = se;
    }
    return VMC_OK;
}

static size_t main_smem(const vmc_ctx* h, int K, size_t at_bytes) {
    return (size_t)h->npf * K * at_bytes * 2 + (size_t)h->M * 4 + 16 * 64;
}

template <int K>
static int apply_S_dispatch(vmc_ctx* h, const double* V, double* out, double shift, int store, cudaStream_t st) {
    // vectors that do not fit the shared-memory image together are split
    // into groups (each group streams the store once)
    if (K > 1) {
        const size_t at = (store == VMC_STORE_FP64 || store == VMC_STORE_FP32) ? 8 : 4;
        // (the sorted BF16 product holds no image: it takes all K at once)
        const bool sorted_all = store == VMC_STORE_BF16 && product_path(h, K) == VMC_PATH_SORTED &&
                                sorted_usable<K>(h);
        if (!sorted_all && main_smem(h, K, at) > h->smem_optin) {
            constexpr int H = K > 1 ? K / 2 : 1;
            int rc = apply_S_dispatch<H>(h, V, out, shift, store, st);
            if (rc) return rc;
            return apply_S_dispatch<H>(h, V + (size_t)H * h->nv, out + (size_t)H * h->nv, shift, store, st);
        }
    }
    const int kind = store_kind(store);
    if (kind < 0) return VMC_ERR_INVALID_ARG;
    if (!store_ptr(h, kind)) return VMC_ERR_STATE;
    int rc0 = ensure_obar(h, kind, st);
    if (rc0) return rc0;
    switch (store) {
        case VMC_STORE_FP64:
            return apply_S_impl<double, double, K>(h, h->d_pf64, kind, V, out, shift, nullptr, nullptr, nullptr, st);
        case VMC_STORE_FP32:
            return apply_S_impl<float, double, K>(h, h->d_pf32, kind, V, out, shift, nullptr, nullptr, nullptr, st);
        case VMC_STORE_BF16:
        case VMC_STORE_FP32_F32ACC: {
            const void* src = store == VMC_STORE_BF16 ? (const void*)h->d_pf16 : (const void*)h->d_pf32;
            if (!src) return VMC_ERR_STATE;
            const int64_t n = h->nv * K;
            k_cast<float><<<kNumPart, 256, 0, st>>>(V, h->d_b32, n, 1.0); h->n_launch++;
            VCK(cudaGetLastError());
            int rc = store == VMC_STORE_BF16
                         ? apply_S_impl<__nv_bfloat16, float, K>(h, src, kind, h->d_b32, h->d_q32, shift, nullptr,
                                                                 nullptr, nullptr, st)
                         : apply_S_impl<float, float, K>(h, src, kind, h->d_b32, h->d_q32, shift, nullptr, nullptr,
                                                         nullptr, st);
            if (rc) return rc;
            // widen back to FP64
            VCK(cudaMemsetAsync(out, 0, sizeof(double) * n, st));
            k_axpy_to64<float><<<kNumPart, 256, 0, st>>>(out, h->d_q32, 1.0, n); h->n_launch++;
            VCK(cudaGetLastError());
            return VMC_OK;
        }
        default:
            return VMC_ERR_INVALID_ARG;
    }
}

extern "C" int sr_apply_S(vmc_handle h, const double* V, double* out, int k, double shift, int store, void* stream) {
    if (!h || !V || !out || k < 1 || k > kMaxK || k == 3) return VMC_ERR_INVALID_ARG;
    if (h->n_s == 0) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    switch (k) {
        case 1: rc = apply_S_dispatch<1>(h, V, out, shift, store, st); break;
        case 2: rc = apply_S_dispatch<2>(h, V, out, shift, store, st); break;
        default: rc = apply_S_dispatch<4>(h, V, out, shift, store, st); break;
    }
    if (rc) return rc;
    return read_status(h, st);   // a staged wait that ran out (synchronizes the stream)
}

extern "C" int vmc_set_product_path(vmc_handle h, int path) {
    if (!h || path < VMC_PATH_AUTO || path > VMC_PATH_COMPACT) return VMC_ERR_INVALID_ARG;
    h->path = path;
    return VMC_OK;
}

extern "C" int vmc_set_auto_paths(vmc_handle h, int path, int path4) {
    if (!h || path < VMC_PATH_SORTED || path > VMC_PATH_COMPACT || path4 < VMC_PATH_SORTED ||
        path4 > VMC_PATH_COMPACT)
        return VMC_ERR_INVALID_ARG;
    h->auto_path = path;
    h->auto_path4 = path4;
    return VMC_OK;
}

// time `reps` BF16 products of K vectors on path `path`; ms < 0 if the path
// does not apply
template <int K>
static int time_path(vmc_ctx* h, int path, int reps, cudaStream_t st, double* ms) {
    *ms = -1.0;
    if (path == VMC_PATH_FUSED && (K != 1 || !fused_usable(h))) return VMC_OK;
    if (path == VMC_PATH_COMPACT && (K != 1 || !compact_usable(h) || !sorted_usable<1>(h))) return VMC_OK;
    if (path == VMC_PATH_SORTED && !sorted_usable<K>(h)) return VMC_OK;
    if (path == VMC_PATH_STAGED && (K > 2 || !h->use_stream)) return VMC_OK;
    const int saved = h->path;
    h->path = path;
    const int64_t n = h->nv * K;
    // a zero vector: the passes do the same work for any input
    if (cudaMemsetAsync(h->d_b32, 0, sizeof(float) * n, st) != cudaSuccess) return VMC_ERR_CUDA;
    int rc = apply_S_impl<__nv_bfloat16, float, K>(h, h->d_pf16, 2, h->d_b32, h->d_q32, 1e-3, nullptr, nullptr,
                                                  nullptr, st);   // warm-up (builds the path's copies)
    cudaEvent_t e0 = h->get_event(), e1 = h->get_event();
    if (!rc) rc = cudaEventRecord(e0, st) == cudaSuccess ? VMC_OK : VMC_ERR_CUDA;
    for (int r = 0; r < reps && !rc; ++r)
        rc = apply_S_impl<__nv_bfloat16, float, K>(h, h->d_pf16, 2, h->d_b32, h->d_q32, 1e-3, nullptr, nullptr,
                                                  nullptr, st);
    if (!rc) rc = cudaEventRecord(e1, st) == cudaSuccess ? VMC_OK : VMC_ERR_CUDA;
    float t = 0.f;
    if (!rc) rc = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess
                      ? VMC_OK : VMC_ERR_CUDA;
    h->ev_pool.push_back(e0);
    h->ev_pool.push_back(e1);
    h->path = saved;
    if (rc == VMC_ERR_UNSUPPORTED) return VMC_OK;
    if (!rc) *ms = (double)t / reps;
    return rc;
}

extern "C" int sr_autotune(vmc_handle h, int reps, vmc_tune_info* info, void* stream) {
    if (!h || reps < 1) return VMC_ERR_INVALID_ARG;
    if (h->n_s == 0 || !h->d_pf16) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_obar(h, 2, st);
    if (rc) return rc;
    vmc_tune_info inf{};
    double best = -1.0, best4 = -1.0;
    inf.path = VMC_PATH_SORTED;
    inf.path4 = VMC_PATH_SORTED;
    for (int p = VMC_PATH_SORTED; p <= VMC_PATH_COMPACT; ++p) {
        double ms = -1.0, ms4 = -1.0;
        if ((rc = time_path<1>(h, p, reps, st, &ms))) return rc;
        if ((rc = time_path<4>(h, p, reps, st, &ms4))) return rc;
        inf.ms[p] = ms;
        inf.ms4[p] = ms4;
        if (ms > 0 && (best < 0 || ms < best)) { best = ms; inf.path = p; }
        if (ms4 > 0 && (best4 < 0 || ms4 < best4)) { best4 = ms4; inf.path4 = p; }
    }
    h->auto_path = inf.path;
    h->auto_path4 = inf.path4;
    if (info) *info = inf;
    return VMC_OK;
}

extern "C" int sr_set_inner_tol(vmc_handle h, double floor) {
    if (!h || !(floor >= 0.0) || floor >= 1.0) return VMC_ERR_INVALID_ARG;
    h->itol_floor = floor;
    return VMC_OK;
}

extern "C" int vmc_set_wait_limit(vmc_handle h, uint32_t tries) {
    if (!h) return VMC_ERR_INVALID_ARG;
    h->wait_limit = tries;
    return VMC_OK;
}

// ---------------------------------------------------------------------------
// conjugate gradient
// ---------------------------------------------------------------------------

// CG on (S + shift I) x = b over store `s_pf` (ST) with vectors of type VT;
// b, x, r, p, q are device vectors of VT.  Returns iterations in *iters.
template <typename ST, typename VT>
static int cg_loop(vmc_ctx* h, const void* s_pf, int kind, const VT* b, VT* x, VT* r, VT* p, VT* q,
                   double shift, double tol, int max_iter, int* iters, cudaStream_t st) {
    const int64_t n = h->nv;
    const double* Obar = h->d_Obar[kind];
    const VT* ObarV = sizeof(VT) == 8 ? (const VT*)h->d_Obar[kind] : (const VT*)h->d_Obar32[kind];
    double* pp_part = h->part(2);    // |p|^2 partials (the first from k_cg_init)
    double* pAp_part = h->part(3);
    double* rr_part = h->part(4);
    double* obp_part = h->part(5);
    double* tt_part = h->part(6);
    const int vg = vgrid(h, 1);
    k_cg_init<VT><<<vg, 256, 0, st>>>(b, x, r, p, n, pp_part); h->n_launch++;
    k_cg_start<<<1, 32, 0, st>>>(pp_part, vg, h->d_scal, tol, h->d_stop); h->n_launch++;
    k_dot_part<double, VT, 1><<<vg, 256, 0, st>>>(Obar, p, n, obp_part, h->d_stop); h->n_launch++;
    VCK(cudaGetLastError());
    int done = 0;
    *iters = 0;
    if (max_iter <= 0) return VMC_OK;
    // centered sorted product with the fused update: gather, scatter, x/r, p
    bool fused = false, single = false;
    if constexpr (sizeof(ST) == 2 && sizeof(VT) == 4) {
        const int path = product_path(h, 1);
        single = path == VMC_PATH_FUSED && fused_usable(h);
        fused = single || ((path == VMC_PATH_SORTED || path == VMC_PATH_FUSED || path == VMC_PATH_COMPACT) &&
                           sorted_usable<1>(h));
    }
    if (fused && h->ncp > 0) VCK(cudaMemsetAsync(h->d_corrraw, 0, sizeof(float) * h->ncp, st));
    // the two updates as one cooperative launch when the update grid is co-resident
    bool coop = false;
    // one pass of the update grid covers the vectors: the register-resident form
    const bool one_pass = (int64_t)vg * 256 * 4 >= n;
    if constexpr (sizeof(VT) == 4) {
        if (fused && h->use_coop_update && h->coop_launch) {
            int per = 0;
            if (one_pass) VCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cg_fxrp1<float>, 256, 0));
            else VCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cg_fxrp<float>, 256, 0));
            coop = (int64_t)per * h->nsm >= vg;
        }
    }
    while (!done) {
        for (int j = 0; j < kChunk; ++j) {
            if (fused) {
                if constexpr (sizeof(ST) == 2 && sizeof(VT) == 4) {
                    int rc = single ? launch_fused(h, p, h->d_invC32, obp_part, (float*)h->d_T, h->d_stop, st, tt_part,
                                                   true)
                                   : launch_sorted<1>(h, p, h->d_invC32, obp_part, (float*)h->d_T, h->d_stop, st,
                                                      tt_part, true);
                    if (rc) return rc;
                    CgFusedArgs<float> f{};
                    f.x = x; f.r = r; f.p = p;
                    f.pf_raw = (const float*)h->d_pfraw;
                    f.corr_raw = (float*)h->d_corrraw;
                    f.invC = h->d_invC32;
                    f.n = n; f.ncp = h->ncp;
                    f.inv_n = 1.0 / (double)h->n_s;
                    f.shift = shift;
                    f.tt_part = tt_part; f.ntt = single ? h->last_fused_grid : h->last_gather_grid;
                    f.pp_part = pp_part; f.npp = vg;
                    f.scal = h->d_scal;
                    f.rr_part = rr_part;
                    f.stop = h->d_stop;
                    if (coop) {
                        // both updates in one cooperative launch (a grid barrier between them)
                        const float* ob = (const float*)ObarV;
                        int* stp = h->d_stop;
                        int mi = max_iter;
                        void* args[] = {&f, &ob, &obp_part, &stp, &mi};
                        VCK(cudaLaunchCooperativeKernel(one_pass ? (const void*)k_cg_fxrp1<float>
                                                                 : (const void*)k_cg_fxrp<float>,
                                                        dim3(vg), dim3(256), args, 0, st));
                        h->n_launch++;
                        VCK(cudaGetLastError());
                        continue;
                    }
                    k_cg_fxr<float><<<vg, 256, 0, st>>>(f); h->n_launch++;
                }
            } else {
                int rc = apply_S_impl<ST, VT, 1>(h, s_pf, kind, p, q, shift, h->d_stop, obp_part, pAp_part, st);
                if (rc) return rc;
                k_cg_xr<VT><<<vg, 256, 0, st>>>(x, r, p, q, n, pAp_part, vg, h->d_scal, rr_part, h->d_stop); h->n_launch++;
            }
            k_cg_p<VT><<<vg, 256, 0, st>>>(r, p, n, rr_part, vg, h->d_scal, ObarV, obp_part, pp_part,
                                           h->d_stop, max_iter); h->n_launch++;
            VCK(cudaGetLastError());
        }
        VCK(cudaMemcpyAsync(h->h_pinned, h->d_scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
        VCK(cudaMemcpyAsync(h->h_pinned + 8, h->d_stop, sizeof(int), cudaMemcpyDeviceToHost, st));
        VCK(cudaMemcpyAsync(h->h_pinned + 9, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
        VCK(cudaStreamSynchronize(st));
        int stop, status;
        memcpy(&stop, h->h_pinned + 8, sizeof(int));
        memcpy(&status, h->h_pinned + 9, sizeof(int));
        if (status & ST_TIMEOUT) {
            VCK(cudaMemsetAsync(h->d_status, 0, sizeof(int), st));
            set_err("a staged wait in the S product ran out");
            return VMC_ERR_TIMEOUT;
        }
        *iters = (int)h->h_pinned[CG_IT];
        if (stop) done = 1;
    }
    return VMC_OK;
}

// y = g - (S + shift I) x with FP64 accumulation over store s_pf (ST = double
// or float); returns |y|^2 through the host.
template <typename ST>
static int residual64(vmc_ctx* h, const void* s_pf, int kind, const double* g, const double* x, double* y,
                      double shift, double* rr, cudaStream_t st) {
    int rc = apply_S_impl<ST, double, 1>(h, s_pf, kind, x, h->d_t64, shift, nullptr, nullptr, nullptr, st);
    if (rc) return rc;
    k_sub<<<kNumPart, 256, 0, st>>>(g, h->d_t64, y, h->nv, h->part(6)); h->n_launch++;
    VCK(cudaGetLastError());
    std::vector<double> parts(kNumPart);
    VCK(cudaMemcpyAsync(parts.data(), h->part(6), sizeof(double) * kNumPart, cudaMemcpyDeviceToHost, st));
    VCK(cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : parts) s += v;
    *rr = s;
    return VMC_OK;
}

static double host_norm2(vmc_ctx* h, const double* v, cudaStream_t st, int* rc) {
    k_dot_part<double, double, 1><<<kNumPart, 256, 0, st>>>(v, v, h->nv, h->part(7), nullptr); h->n_launch++;
    std::vector<double> parts(kNumPart);
    if (cudaMemcpyAsync(parts.data(), h->part(7), sizeof(double) * kNumPart, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        *rc = VMC_ERR_CUDA;
        return 0.0;
    }
    double s = 0.0;
    for (double x : parts) s += x;
    *rc = VMC_OK;
    return s;
}

static double dot64(vmc_ctx* h, const double* a, const double* b, cudaStream_t st, int* rc) {
    k_dot_part<double, double, 1><<<kNumPart, 256, 0, st>>>(a, b, h->nv, h->part(7), nullptr); h->n_launch++;
    std::vector<double> parts(kNumPart);
    if (cudaMemcpyAsync(parts.data(), h->part(7), sizeof(double) * kNumPart, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        *rc = VMC_ERR_CUDA;
        return 0.0;
    }
    double s = 0.0;
    for (double v : parts) s += v;
    *rc = VMC_OK;
    return s;
}

// z = M^{-1} r: the inner low-precision CG on (S_lowp + shift I) with the
// right-hand side scaled to unit norm, to relative tolerance itol.
static int inner_block(vmc_ctx* h, const double* r, double rnorm, double* z, double shift, double itol,
                       int max_iter, int* iters, cudaStream_t st);

static int inner_solve(vmc_ctx* h, int mode, const double* r, double rnorm, double* z, double shift, double itol,
                       int max_iter, int* iters, cudaStream_t st) {
    if (mode == VMC_CG_BLOCK4) {
        int rc = inner_block(h, r, rnorm, z, shift, itol, max_iter, iters, st);
        if (rc || *iters > 0) return rc;
        mode = VMC_CG_MIXED;   // no block step possible: one-vector inner CG
    }
    k_cast<float><<<kNumPart, 256, 0, st>>>(r, h->d_b32, h->nv, 1.0 / rnorm); h->n_launch++;
    VCK(cudaGetLastError());
    int rc = (mode == VMC_CG_MIXED || mode == VMC_CG_MIXED64)
                 ? cg_loop<__nv_bfloat16, float>(h, h->d_pf16, 2, h->d_b32, h->d_x32, h->d_r32, h->d_p32,
                                                h->d_q32, shift, itol, max_iter, iters, st)
                 : cg_loop<float, float>(h, h->d_pf32, 1, h->d_b32, h->d_x32, h->d_r32, h->d_p32, h->d_q32,
                                        shift, itol, max_iter, iters, st);
    if (rc) return rc;
    VCK(cudaMemsetAsync(z, 0, sizeof(double) * h->nv, st));
    k_axpy_to64<float><<<kNumPart, 256, 0, st>>>(z, h->d_x32, rnorm, h->nv); h->n_launch++;
    VCK(cudaGetLastError());
    return VMC_OK;
}

// z = M^{-1} r by enlarged block CG on the BF16 operator: the unit-norm
// right-hand side split into four parameter-group columns, O'Leary's block
// recurrences (alpha = (P^T Q)^{-1} R^T R, beta = (R^T R)^{-1} R_new^T R_new),
// stopped when the residual of the column sum, |sum_j R_j|^2 = sum of the
// entries of R^T R, meets itol; z = |r| sum_j X_j.  The iteration runs on the
// device (bcg.cu): per step the four-vector product, the P^T Q Gram with the
// alpha solve, the X/R update with the new R^T R Gram, the beta solve with
// the stopping test, and the new directions with their Obar . P partials
// (the next product's centering); the host reads the state every kChunk
// steps.
static int inner_block(vmc_ctx* h, const double* r, double rnorm, double* z, double shift, double itol,
                       int max_iter, int* iters, cudaStream_t st) {
    const int64_t n = h->nv;
    const size_t npart = (size_t)kNumPart * kMaxK * 16;
    if (!h->d_bcg) VCK(h->alloc(&h->d_bcg, npart + (sizeof(BcgState) + 7) / 8));
    double* gpart = h->d_bcg;
    BcgState* S = (BcgState*)(h->d_bcg + npart);
    double* obp_part = h->part(5);
    float *X = h->d_x32, *R = h->d_r32, *P = h->d_p32, *Q = h->d_q32;
    const int vg = vgrid(h, 1), vg4 = vgrid(h, 4);
    *iters = 0;
    k_cast<float><<<kNumPart, 256, 0, st>>>(r, h->d_b32, n, 1.0 / rnorm);
    k_bcg_split<<<vg, 256, 0, st>>>(h->d_b32, R, n, h->ncp, h->corr_off[h->ncorr / 2], h->d_pq_of, h->ns);
    h->n_launch += 2;
    VCK(cudaMemsetAsync(X, 0, sizeof(float) * 4 * n, st));
    VCK(cudaMemcpyAsync(P, R, sizeof(float) * 4 * n, cudaMemcpyDeviceToDevice, st));
    VCK(cudaMemsetAsync(h->d_stop, 0, sizeof(int), st));
    k_bcg_gram<<<vg, 256, 0, st>>>(R, R, n, gpart, nullptr);
    k_bcg_start<<<1, 256, 0, st>>>(gpart, vg, S, itol);
    k_dot_part<double, float, 4><<<vg4, 256, 0, st>>>(h->d_Obar[2], P, n, obp_part, nullptr);
    h->n_launch += 3;
    VCK(cudaGetLastError());
    // an inner solve that has not met itol after kBlockInnerMax steps returns
    // what it has: the flexible outer iteration takes any preconditioner
    max_iter = std::min(max_iter, kBlockInnerMax);
    for (int done = 0; !done;) {
        for (int j = 0; j < kChunk; ++j) {
            int rc = apply_S_impl<__nv_bfloat16, float, 4>(h, h->d_pf16, 2, P, Q, shift, h->d_stop, obp_part, nullptr, st);
            if (rc) return rc;
            k_bcg_gram<<<vg, 256, 0, st>>>(P, Q, n, gpart, h->d_stop);
            k_bcg_alpha<<<1, 256, 0, st>>>(gpart, vg, S, h->d_stop);
            k_bcg_step<<<vg, 256, 0, st>>>(X, R, P, Q, S, n, gpart, h->d_stop);
            k_bcg_beta<<<1, 256, 0, st>>>(gpart, vg, S, h->d_stop, max_iter);
            k_bcg_dir<<<vg4, 256, 0, st>>>(P, R, S, h->d_Obar[2], n, obp_part, h->d_stop);
            h->n_launch += 5;
            VCK(cudaGetLastError());
        }
        BcgState hs;
        int stop = 0;
        VCK(cudaMemcpyAsync(&hs, S, sizeof(hs), cudaMemcpyDeviceToHost, st));
        VCK(cudaMemcpyAsync(&stop, h->d_stop, sizeof(int), cudaMemcpyDeviceToHost, st));
        VCK(cudaStreamSynchronize(st));
        if (stop || hs.it >= max_iter) {
            done = 1;
            *iters = hs.steps > 0 ? hs.it : 0;   // 0: no block step was possible
        }
    }
    VCK(cudaMemsetAsync(z, 0, sizeof(double) * n, st));
    for (int j = 0; j < 4; ++j) {
        k_axpy_to64<float><<<kNumPart, 256, 0, st>>>(z, X + (size_t)j * n, rnorm, n);
        h->n_launch++;
    }
    VCK(cudaGetLastError());
    return VMC_OK;
}

// Flexible conjugate gradient (Notay, SIAM J. Sci. Comput. 22, 2000; one
// retained direction) on (S + shift I) x = g.  The outer product streams the
// FP32 store with FP64 accumulation; the preconditioner is the inner BF16 (or
// FP32) CG solve, whose error varies from step to step - hence the flexible
// beta = -alpha (z_new . q) / (z . r).
static int fcg_mixed(vmc_ctx* h, const double* g, double shift, double tol, int max_iter, int mode, double* x,
                     double gn2, vmc_cg_info* inf, cudaStream_t st) {
    const int64_t n = h->nv;
    double* r = h->d_r64;
    double* z = h->d_x64;
    double* p = h->d_p64;
    double* q = h->d_q64;
    int rc = VMC_OK;
    VCK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    VCK(cudaMemcpyAsync(r, g, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    double rr = gn2;
    const double target = tol * tol * gn2;
    // inner accuracy beyond about ten percent buys little: the BF16 operator's
    // own error limits what one preconditioner application can contribute
    // default floors: BF16 inner solves 0.1 (a sweep of 0.003 .. 0.3 on the
    // 8x8 / 2x3 workload measured it fastest: fewer inner products than 3e-2 at
    // one more outer step), FP32 inner solves 1e-3
    const double itol_floor = h->itol_floor > 0.0 ? h->itol_floor : mode == VMC_CG_FP32 ? 1e-3 : 0.1;
    int used = 0;
    if (rr == 0.0) { inf->true_rel_residual = 0.0; return VMC_OK; }
    double rn = std::sqrt(rr);
    int it = 0;
    rc = inner_solve(h, mode, r, rn, z, shift, std::max(itol_floor, 0.5 * std::sqrt(target / rr)), max_iter, &it, st);
    if (rc) return rc;
    used += it;
    VCK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    double zr = dot64(h, z, r, st, &rc);
    if (rc) return rc;
    // the outer operator: the FP64 store (MIXED64) or the FP32 store with
    // FP64 accumulation
    const bool outer64 = mode == VMC_CG_MIXED64;
    for (int outer = 0; outer < 200; ++outer) {
        rc = outer64 ? apply_S_impl<double, double, 1>(h, h->d_pf64, 0, p, q, shift, nullptr, nullptr, nullptr, st)
                     : apply_S_impl<float, double, 1>(h, h->d_pf32, 1, p, q, shift, nullptr, nullptr, nullptr, st);
        if (rc) return rc;
        inf->residual_products++;
        double pq = dot64(h, p, q, st, &rc);
        if (rc) return rc;
        if (!(pq > 0.0)) break;
        const double alpha = zr / pq;
        k_axpby<<<kNumPart, 256, 0, st>>>(alpha, p, 1.0, x, n); h->n_launch++;
        k_axpby<<<kNumPart, 256, 0, st>>>(-alpha, q, 1.0, r, n); h->n_launch++;
        VCK(cudaGetLastError());
        rr = dot64(h, r, r, st, &rc);
        if (rc) return rc;
        inf->refinements++;
        if (rr <= target || used >= max_iter) break;
        rn = std::sqrt(rr);
        rc = inner_solve(h, mode, r, rn, z, shift, std::max(itol_floor, 0.5 * std::sqrt(target / rr)),
                         max_iter - used, &it, st);
        if (rc) return rc;
        used += it;
        const double zq = dot64(h, z, q, st, &rc);
        if (rc) return rc;
        const double zr_new = dot64(h, z, r, st, &rc);
        if (rc) return rc;
        const double beta = -alpha * zq / zr;
        k_axpby<<<kNumPart, 256, 0, st>>>(1.0, z, beta, p, n); h->n_launch++;
        VCK(cudaGetLastError());
        zr = zr_new;
    }
    // true residual of the returned x, FP64 accumulation over the outer store
    double rt = 0.0;
    rc = outer64 ? residual64<double>(h, h->d_pf64, 0, g, x, h->d_r64, shift, &rt, st)
                 : residual64<float>(h, h->d_pf32, 1, g, x, h->d_r64, shift, &rt, st);
    if (rc) return rc;
    inf->residual_products++;
    inf->iterations = used;
    inf->true_rel_residual = std::sqrt(rt / gn2);
    return VMC_OK;
}

extern "C" int sr_cg_solve(vmc_handle h, const double* g, double shift, double tol, int max_iter, int mode, double* x,
                           vmc_cg_info* info, void* stream) {
    if (!h || !g || !x || !(tol > 0) || max_iter < 1) return VMC_ERR_INVALID_ARG;
    if (h->n_s == 0) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    vmc_cg_info inf{};
    int rc = VMC_OK;
    const double gn2 = host_norm2(h, g, st, &rc);
    if (rc) return rc;
    if (mode == VMC_CG_FP64) {
        if (!h->d_pf64) return VMC_ERR_STATE;
        rc = ensure_obar(h, 0, st);
        if (rc) return rc;
        int it = 0;
        rc = cg_loop<double, double>(h, h->d_pf64, 0, g, h->d_x64, h->d_r64, h->d_p64, h->d_q64, shift, tol,
                                     max_iter, &it, st);
        if (rc) return rc;
        VCK(cudaMemcpyAsync(x, h->d_x64, sizeof(double) * h->nv, cudaMemcpyDeviceToDevice, st));
        double rr = 0.0;
        rc = residual64<double>(h, h->d_pf64, 0, g, x, h->d_r64, shift, &rr, st);
        if (rc) return rc;
        inf.iterations = it;
        inf.residual_products = 1;
        inf.true_rel_residual = gn2 > 0 ? std::sqrt(rr / gn2) : 0.0;
    } else if (mode == VMC_CG_MIXED || mode == VMC_CG_FP32 || mode == VMC_CG_BLOCK4 || mode == VMC_CG_MIXED64) {
        if (!h->d_pf32 || !h->d_pf16) return VMC_ERR_STATE;
        if (mode == VMC_CG_MIXED64) {
            if (!h->d_pf64) return VMC_ERR_STATE;
            rc = ensure_obar(h, 0, st);
            if (rc) return rc;
        }
        if (mode == VMC_CG_BLOCK4) {
            // the four parameter groups must all be non-empty
            const int64_t split = h->ncorr >= 2 ? h->corr_off[h->ncorr / 2] : 0;
            if (split <= 0 || split >= h->ncp || h->ns < 2) {
                set_err("block CG needs at least two correlator blocks and two sites");
                return VMC_ERR_UNSUPPORTED;
            }
        }
        rc = ensure_obar(h, 1, st);
        if (!rc && mode != VMC_CG_FP32) rc = ensure_obar(h, 2, st);
        if (rc) return rc;
        rc = fcg_mixed(h, g, shift, tol, max_iter, mode, x, gn2, &inf, st);
        if (rc) return rc;
    } else {
        return VMC_ERR_INVALID_ARG;
    }
    inf.converged = inf.true_rel_residual <= tol ? 1 : 0;
    if (info) *info = inf;
    return inf.converged ? VMC_OK : VMC_ERR_NOT_CONVERGED;
}

extern "C" int sr_update(vmc_handle h, const double* y, double tau, int store, double* x0, void* stream) {
    if (!h || !y || !std::isfinite(tau)) return VMC_ERR_INVALID_ARG;
    const int kind = store_kind(store);
    if (kind < 0) return VMC_ERR_INVALID_ARG;
    if (!h->params_set || h->n_s == 0 || !h->obar_ok[kind]) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    k_vec_sum<<<kNumPart, 256, 0, st>>>(h->d_E, h->n_s, h->part(0)); h->n_launch++;
    k_dot_part<double, double, 1><<<kNumPart, 256, 0, st>>>(h->d_Obar[kind], y, h->nv, h->part(1), nullptr);
    h->n_launch++;
    UpdateArgs a{};
    a.C64 = h->d_C64; a.C32 = h->d_C32; a.invC64 = h->d_invC64; a.invC32 = h->d_invC32;
    a.F64 = h->d_F64; a.F32 = h->d_F32; a.pq_of = h->d_pq_of;
    a.y = y;
    a.ncp = h->ncp; a.npf = h->npf; a.M = h->M;
    a.tau = tau; a.inv_n = 1.0 / (double)h->n_s;
    a.e_part = h->part(0); a.ne = kNumPart;
    a.oy_part = h->part(1); a.noy = kNumPart;
    a.x0 = h->d_scal + kScalX0;
    a.status = h->d_status;
    k_sr_update<<<vgrid(h, 1), 256, 0, st>>>(a); h->n_launch++;
    VCK(cudaGetLastError());
    // the stored samples belong to the old parameters
    h->obar_ok[0] = h->obar_ok[1] = h->obar_ok[2] = false;
    h->sorted_ok = h->g_ok = h->corr_ok = false;
    VCK(cudaMemcpyAsync(h->h_pinned + 1, h->d_scal + kScalX0, sizeof(double), cudaMemcpyDeviceToHost, st));
    int rc = read_status(h, st);   // synchronizes the stream
    if (x0) *x0 = h->h_pinned[1];
    return rc;
}

// ---------------------------------------------------------------------------
// rank-local sums for a sample-sharded solve
// ---------------------------------------------------------------------------

extern "C" int sr_local_moments(vmc_handle h, double* sumO, double* sumEO, double* scal, int store, void* stream) {
    if (!h || !sumO || !sumEO || !scal) return VMC_ERR_INVALID_ARG;
    const int kind = store_kind(store);
    if (kind < 0) return VMC_ERR_INVALID_ARG;
    if (h->n_s == 0) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = gradient_pass(h, kind, h->d_t64, st);   // Obar[kind], g, E partial sums in part(1)
    if (rc) return rc;
    std::vector<double> parts(kNumPart);
    VCK(cudaMemcpyAsync(parts.data(), h->part(1), sizeof(double) * kNumPart, cudaMemcpyDeviceToHost, st));
    VCK(cudaStreamSynchronize(st));
    double sE = 0.0;
    for (double v : parts) sE += v;
    const double n = (double)h->n_s;
    // sum O = n Obar; sum E O = n g + (sum E) Obar
    k_cast<double><<<kNumPart, 256, 0, st>>>(h->d_Obar[kind], sumO, h->nv, n); h->n_launch++;
    k_cast<double><<<kNumPart, 256, 0, st>>>(h->d_t64, sumEO, h->nv, n); h->n_launch++;
    k_axpby<<<kNumPart, 256, 0, st>>>(sE, h->d_Obar[kind], 1.0, sumEO, h->nv); h->n_launch++;
    VCK(cudaGetLastError());
    scal[0] = sE;
    scal[1] = n;
    return VMC_OK;
}

extern "C" int sr_local_product(vmc_handle h, const double* v, double* out, int store, void* stream) {
    if (!h || !v || !out) return VMC_ERR_INVALID_ARG;
    if (store != VMC_STORE_FP64 && store != VMC_STORE_FP32) return VMC_ERR_INVALID_ARG;
    const int kind = store_kind(store);
    if (h->n_s == 0 || !store_ptr(h, kind) || !h->obar_ok[kind]) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    // out = S v with shift 0 (uncentered pass, covariance term in the finalize),
    // then back to the plain sum; Obar . v is left in part(0) by the product
    int rc = kind == 0 ? apply_S_impl<double, double, 1>(h, h->d_pf64, kind, v, out, 0.0, nullptr, nullptr, nullptr, st)
                       : apply_S_impl<float, double, 1>(h, h->d_pf32, kind, v, out, 0.0, nullptr, nullptr, nullptr, st);
    if (rc) return rc;
    k_uncenter<<<kNumPart, 256, 0, st>>>(out, h->d_Obar[kind], h->part(0), vgrid(h, 1), (double)h->n_s, h->nv);
    h->n_launch++;
    VCK(cudaGetLastError());
    return VMC_OK;
}

// ---------------------------------------------------------------------------
// accelerated linear method (Sec. II.B)
// ---------------------------------------------------------------------------
static int lm_ensure(vmc_ctx* h) {
    if (h->d_lmL64) return VMC_OK;
    // the factors as sparse matrices: nonzeros of each L^mu (R^mu) in row order
    const size_t n2 = (size_t)h->ns * h->ns;
    std::vector<int> ptr[2], idx[2];
    std::vector<double> val[2];
    for (int side = 0; side < 2; ++side) {
        const std::vector<double>& F = side == 0 ? h->lm_L : h->lm_R;
        ptr[side].push_back(0);
        for (int mu = 0; mu < h->lm_nmu; ++mu) {
            for (size_t t = 0; t < n2; ++t) {
                const double v = F[(size_t)mu * n2 + t];
                if (v != 0.0) { idx[side].push_back((int)t); val[side].push_back(v); }
            }
            ptr[side].push_back((int)idx[side].size());
        }
    }
    std::vector<float> L32(val[0].begin(), val[0].end()), R32(val[1].begin(), val[1].end());
    VCK(h->alloc(&h->d_lmL64, val[0].size()));
    VCK(h->alloc(&h->d_lmR64, val[1].size()));
    VCK(h->alloc(&h->d_lmL32, val[0].size()));
    VCK(h->alloc(&h->d_lmR32, val[1].size()));
    VCK(h->alloc(&h->d_lmLptr, ptr[0].size()));
    VCK(h->alloc(&h->d_lmRptr, ptr[1].size()));
    VCK(h->alloc(&h->d_lmLidx, idx[0].size()));
    VCK(h->alloc(&h->d_lmRidx, idx[1].size()));
    VCK(h->alloc(&h->d_lmXt, (size_t)h->M * h->M));
    VCK(h->alloc(&h->d_lmxc, (size_t)std::max<int64_t>(h->ncp, 1)));
    auto up = [](void* d, const void* s, size_t b) { return b ? cudaMemcpy(d, s, b, cudaMemcpyHostToDevice) : cudaSuccess; };
    VCK(up(h->d_lmL64, val[0].data(), val[0].size() * sizeof(double)));
    VCK(up(h->d_lmR64, val[1].data(), val[1].size() * sizeof(double)));
    VCK(up(h->d_lmL32, L32.data(), L32.size() * sizeof(float)));
    VCK(up(h->d_lmR32, R32.data(), R32.size() * sizeof(float)));
    VCK(up(h->d_lmLptr, ptr[0].data(), ptr[0].size() * sizeof(int)));
    VCK(up(h->d_lmRptr, ptr[1].data(), ptr[1].size() * sizeof(int)));
    VCK(up(h->d_lmLidx, idx[0].data(), idx[0].size() * sizeof(int)));
    VCK(up(h->d_lmRidx, idx[1].data(), idx[1].size() * sizeof(int)));
    return VMC_OK;
}

template <typename R>
static int lm_launch(vmc_ctx* h, const double* x, double* Hx, double* Sx, const R* pf, const R* Lf,
                     const R* Rf, cudaStream_t st) {
    R* Xt = (R*)h->d_lmXt;
    R* xc = (R*)h->d_lmxc;
    const int64_t nprep = (int64_t)h->M * h->M + h->ncp;
    k_lm_prep<R><<<(unsigned)std::min<int64_t>((nprep + 255) / 256, 4 * h->nsm), 256, 0, st>>>(h->pb, x, Xt, xc);
    h->n_launch++;
    LmArgs a{};
    a.pb = h->pb;
    a.n_s = h->n_s;
    a.s_occ = h->d_socc; a.Nst = h->Nst;
    a.s_cidx = h->d_cidx; a.ncst = h->ncst;
    a.pf = pf; a.Pst = h->Pst;
    a.x = x; a.Xt = Xt; a.xc = xc;
    a.n_mu = h->lm_nmu; a.c0 = h->lm_c0;
    a.Lptr = h->d_lmLptr; a.Lidx = h->d_lmLidx; a.Lval = Lf;
    a.Rptr = h->d_lmRptr; a.Ridx = h->d_lmRidx; a.Rval = Rf;
    a.inv_n = 1.0 / (double)h->n_s;
    a.Hx = Hx; a.Sx = Sx;
    a.XS = h->N + 1; a.GS = h->N + 1;
    a.warp_bytes = (int)lm_warp_bytes(h->N, h->M, h->ns, h->lm_nmu, h->ncorr, (int)sizeof(R));
    if ((size_t)a.warp_bytes > h->smem_optin) {
        set_err("linear-method product: per-sample workspace exceeds shared memory");
        return VMC_ERR_UNSUPPORTED;
    }
    const int wpb = (int)std::min<size_t>(8, h->smem_optin / (size_t)a.warp_bytes);
    const size_t smem = (size_t)wpb * a.warp_bytes;
    VCK(cudaFuncSetAttribute(k_lm_apply<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    VCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lm_apply<R>, 32 * wpb, smem));
    const int64_t need = (h->n_s + wpb - 1) / wpb;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)h->nsm * std::max(per_sm, 1)));
    k_lm_apply<R><<<grid, 32 * wpb, smem, st>>>(a);
    h->n_launch++;
    VCK(cudaGetLastError());
    return VMC_OK;
}

extern "C" int lm_apply(vmc_handle h, const double* x, double* Hx, double* Sx, int store, void* stream) {
    if (!h || !x || !Hx) return VMC_ERR_INVALID_ARG;
    if (store != VMC_STORE_FP64 && store != VMC_STORE_FP32) return VMC_ERR_INVALID_ARG;
    if (h->n_s == 0 || !h->params_set) return VMC_ERR_STATE;
    if (store == VMC_STORE_FP64 ? !h->d_pf64 : !h->d_pf32) return VMC_ERR_STATE;
    int rc = lm_ensure(h);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nb = sizeof(double) * (size_t)(h->nv + 1);
    VCK(cudaMemsetAsync(Hx, 0, nb, st));
    if (Sx) VCK(cudaMemsetAsync(Sx, 0, nb, st));
    return store == VMC_STORE_FP64
               ? lm_launch<double>(h, x, Hx, Sx, h->d_pf64, h->d_lmL64, h->d_lmR64, st)
               : lm_launch<float>(h, x, Hx, Sx, h->d_pf32, h->d_lmL32, h->d_lmR32, st);
}

namespace {

// lowest eigenpair of h c = theta s c (m x m symmetric, s positive
// definite): s = L L^T, A = L^{-1} h L^{-T}, cyclic Jacobi on A, c = L^{-T} y
bool small_gen_eig(int m, const std::vector<double>& hm, const std::vector<double>& sm, double* theta,
                   std::vector<double>& c) {
    std::vector<double> L(sm);
    for (int j = 0; j < m; ++j) {
        double d = L[j * m + j];
        for (int k = 0; k < j; ++k) d -= L[j * m + k] * L[j * m + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        L[j * m + j] = d;
        for (int i = j + 1; i < m; ++i) {
            double v = L[i * m + j];
            for (int k = 0; k < j; ++k) v -= L[i * m + k] * L[j * m + k];
            L[i * m + j] = v / d;
        }
        for (int k = j + 1; k < m; ++k) L[j * m + k] = 0.0;
    }
    // B = L^{-1} h (forward substitution per column), A = B L^{-T}
    std::vector<double> B(hm), A((size_t)m * m);
    for (int col = 0; col < m; ++col)
        for (int i = 0; i < m; ++i) {
            double v = B[i * m + col];
            for (int k = 0; k < i; ++k) v -= L[i * m + k] * B[k * m + col];
            B[i * m + col] = v / L[i * m + i];
        }
    for (int row = 0; row < m; ++row)
        for (int i = 0; i < m; ++i) {
            double v = B[row * m + i];
            for (int k = 0; k < i; ++k) v -= A[row * m + k] * L[i * m + k];
            A[row * m + i] = v / L[i * m + i];
        }
    for (int i = 0; i < m; ++i)
        for (int j = i + 1; j < m; ++j) A[i * m + j] = A[j * m + i] = 0.5 * (A[i * m + j] + A[j * m + i]);
    std::vector<double> Q((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) Q[i * m + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) (i == j ? tot : off) += A[i * m + j] * A[i * m + j];
        if (off <= 1e-30 * (tot + off) || off == 0.0) break;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) {
                const double apq = A[p * m + q];
                if (apq == 0.0) continue;
                const double tau = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
                for (int k = 0; k < m; ++k) {
                    const double akp = A[k * m + p], akq = A[k * m + q];
                    A[k * m + p] = cs * akp - sn * akq;
                    A[k * m + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < m; ++k) {
                    const double apk = A[p * m + k], aqk = A[q * m + k];
                    A[p * m + k] = cs * apk - sn * aqk;
                    A[q * m + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < m; ++k) {
                    const double qkp = Q[k * m + p], qkq = Q[k * m + q];
                    Q[k * m + p] = cs * qkp - sn * qkq;
                    Q[k * m + q] = sn * qkp + cs * qkq;
                }
            }
    }
    int lo = 0;
    for (int i = 1; i < m; ++i)
        if (A[i * m + i] < A[lo * m + lo]) lo = i;
    *theta = A[lo * m + lo];
    c.assign(m, 0.0);
    for (int i = m - 1; i >= 0; --i) {   // L^T c = y
        double v = Q[i * m + lo];
        for (int k = i + 1; k < m; ++k) v -= L[k * m + i] * c[k];
        c[i] = v / L[i * m + i];
    }
    return std::isfinite(*theta);
}

}  // namespace

static int lm_dots(vmc_ctx* h, const double* V, int k, const double* u, double* out_host, cudaStream_t st) {
    const int64_t n = h->nv + 1;
    k_lm_dots<<<kNumPart, 256, 0, st>>>(V, h->lm_ld, k, u, n, h->d_lmdot);
    k_lm_dots_reduce<<<1, 64, 0, st>>>(h->d_lmdot, kNumPart, k, h->d_lmdot + (size_t)kNumPart * h->lm_cap);
    h->n_launch += 2;
    VCK(cudaMemcpyAsync(out_host, h->d_lmdot + (size_t)kNumPart * h->lm_cap, sizeof(double) * k,
                        cudaMemcpyDeviceToHost, st));
    VCK(cudaStreamSynchronize(st));
    return VMC_OK;
}

extern "C" int lm_solve(vmc_handle h, double shift_H, double shift_S, double tol, int max_iter, int max_sub,
                        double* x, vmc_lm_info* info, int store, void* stream) {
    if (!h || !x || !(shift_S > 0.0) || !std::isfinite(shift_H) || !(tol > 0.0) || max_iter < 1 || max_sub < 3 ||
        max_sub > 64)
        return VMC_ERR_INVALID_ARG;
    if (store != VMC_STORE_FP64 && store != VMC_STORE_FP32) return VMC_ERR_INVALID_ARG;
    if (h->n_s == 0 || !h->params_set) return VMC_ERR_STATE;
    if (store == VMC_STORE_FP64 ? !h->d_pf64 : !h->d_pf32) return VMC_ERR_STATE;
    int rc = lm_ensure(h);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = h->nv + 1;
    if (h->lm_cap < max_sub) {
        h->lm_cap = max_sub;
        h->lm_ld = round_up(n, 32);
        VCK(h->alloc(&h->d_lmV, (size_t)h->lm_ld * max_sub));
        VCK(h->alloc(&h->d_lmHV, (size_t)h->lm_ld * max_sub));
        VCK(h->alloc(&h->d_lmSV, (size_t)h->lm_ld * max_sub));
        VCK(h->alloc(&h->d_lmW, (size_t)h->lm_ld * 12));
        VCK(h->alloc(&h->d_lmdot, (size_t)(kNumPart + 1) * h->lm_cap + 64));
    }
    const int64_t ld = h->lm_ld;
    double* W = h->d_lmW;
    double *t = W, *Ht = W + ld, *St = W + 2 * ld, *u = W + 3 * ld, *Hu = W + 4 * ld, *Su = W + 5 * ld;
    double *r = W + 6 * ld, *up = W + 7 * ld, *d = W + 8 * ld;
    double* dc = h->d_lmdot + (size_t)(kNumPart + 1) * h->lm_cap;   // 64 coefficients on the device
    double *V = h->d_lmV, *HV = h->d_lmHV, *SV = h->d_lmSV;
    const unsigned vg = (unsigned)vgrid(h, 1);
    auto launch_ok = [&]() { return cudaGetLastError(); };

    // preconditioner: diag(S) + shift_S D
    VCK(cudaMemsetAsync(d, 0, sizeof(double) * n, st));
    {
        LmArgs a{};
        a.pb = h->pb; a.n_s = h->n_s; a.s_occ = h->d_socc; a.Nst = h->Nst; a.s_cidx = h->d_cidx; a.ncst = h->ncst;
        a.pf = store == VMC_STORE_FP64 ? (const void*)h->d_pf64 : (const void*)h->d_pf32;
        a.Pst = h->Pst; a.inv_n = 1.0 / (double)h->n_s;
        const unsigned g = (unsigned)std::min<int64_t>((h->n_s + 7) / 8, 8 * h->nsm);
        if (store == VMC_STORE_FP64) k_lm_diag<double><<<g, 256, 0, st>>>(a, d);
        else k_lm_diag<float><<<g, 256, 0, st>>>(a, d);
        h->n_launch++;
        const double one = 1.0;
        VCK(cudaMemcpyAsync(d, &one, sizeof(double), cudaMemcpyHostToDevice, st));
        VCK(cudaStreamSynchronize(st));
    }
    // start from e_0 (the current wavefunction)
    VCK(cudaMemsetAsync(t, 0, sizeof(double) * n, st));
    {
        const double one = 1.0;
        VCK(cudaMemcpyAsync(t, &one, sizeof(double), cudaMemcpyHostToDevice, st));
        VCK(cudaStreamSynchronize(st));
    }
    std::vector<double> hm((size_t)max_sub * max_sub), sm((size_t)max_sub * max_sub), cv, col(max_sub), row(max_sub);
    int m = 0, iters = 0, restarts = 0;
    bool have_prev = false, conv = false;
    double theta = 0.0, relres = INFINITY;
    auto orthonormalize = [&](double* vec) -> int {
        for (int pass = 0; pass < 2 && m > 0; ++pass) {
            int e = lm_dots(h, V, m, vec, col.data(), st);
            if (e) return e;
            for (int j = 0; j < m; ++j) col[j] = -col[j];
            VCK(cudaMemcpyAsync(dc, col.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
            k_lm_combine<<<vg, 256, 0, st>>>(vec, V, ld, m, dc, n, 1.0); h->n_launch++;
        }
        double nrm2;
        int e = lm_dots(h, vec, 1, vec, &nrm2, st);
        if (e) return e;
        if (!(nrm2 > 0.0) || !std::isfinite(nrm2)) return VMC_ERR_NONFINITE;
        k_axpby<<<vg, 256, 0, st>>>(0.0, vec, 1.0 / std::sqrt(nrm2), vec, n); h->n_launch++;
        return VMC_OK;
    };
    // append column m (vec, H vec, S vec) and extend the projected matrices
    auto append = [&](const double* vec, const double* Hvec, const double* Svec) -> int {
        VCK(cudaMemcpyAsync(V + (size_t)m * ld, vec, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        VCK(cudaMemcpyAsync(HV + (size_t)m * ld, Hvec, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        VCK(cudaMemcpyAsync(SV + (size_t)m * ld, Svec, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        ++m;
        int e;
        if ((e = lm_dots(h, V, m, HV + (size_t)(m - 1) * ld, col.data(), st))) return e;   // V^T H v_new
        if ((e = lm_dots(h, HV, m, V + (size_t)(m - 1) * ld, row.data(), st))) return e;   // (H V)^T v_new
        for (int i = 0; i < m; ++i) hm[(size_t)i * max_sub + (m - 1)] = hm[(size_t)(m - 1) * max_sub + i] = 0.5 * (col[i] + row[i]);
        if ((e = lm_dots(h, V, m, SV + (size_t)(m - 1) * ld, col.data(), st))) return e;
        if ((e = lm_dots(h, SV, m, V + (size_t)(m - 1) * ld, row.data(), st))) return e;
        for (int i = 0; i < m; ++i) sm[(size_t)i * max_sub + (m - 1)] = sm[(size_t)(m - 1) * max_sub + i] = 0.5 * (col[i] + row[i]);
        return VMC_OK;
    };
    auto combine3 = [&](const std::vector<double>& c, int k) -> int {
        VCK(cudaMemcpyAsync(dc, c.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
        k_lm_combine<<<vg, 256, 0, st>>>(u, V, ld, k, dc, n, 0.0);
        k_lm_combine<<<vg, 256, 0, st>>>(Hu, HV, ld, k, dc, n, 0.0);
        k_lm_combine<<<vg, 256, 0, st>>>(Su, SV, ld, k, dc, n, 0.0);
        h->n_launch += 3;
        return VMC_OK;
    };
    for (iters = 1; iters <= max_iter; ++iters) {
        if ((rc = orthonormalize(t))) return rc;
        if ((rc = lm_apply(h, t, Ht, St, store, stream))) return rc;
        // shifts on the parameter block (component 0 untouched)
        k_axpby<<<vg, 256, 0, st>>>(shift_H, t + 1, 1.0, Ht + 1, n - 1);
        k_axpby<<<vg, 256, 0, st>>>(shift_S, t + 1, 1.0, St + 1, n - 1);
        h->n_launch += 2;
        if ((rc = append(t, Ht, St))) return rc;
        std::vector<double> hh((size_t)m * m), ss((size_t)m * m);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                hh[(size_t)i * m + j] = hm[(size_t)i * max_sub + j];
                ss[(size_t)i * m + j] = sm[(size_t)i * max_sub + j];
            }
        if (!small_gen_eig(m, hh, ss, &theta, cv)) {
            set_err("lm_solve: projected overlap not positive definite");
            return VMC_ERR_NONFINITE;
        }
        if ((rc = combine3(cv, m))) return rc;
        k_axpby<<<vg, 256, 0, st>>>(1.0, Hu, 0.0, r, n);
        k_axpby<<<vg, 256, 0, st>>>(-theta, Su, 1.0, r, n);
        h->n_launch += 2;
        double rr, ss2;
        if ((rc = lm_dots(h, r, 1, r, &rr, st))) return rc;
        if ((rc = lm_dots(h, Su, 1, Su, &ss2, st))) return rc;
        relres = std::sqrt(rr) / (std::fabs(theta) * std::sqrt(ss2));
        if (relres <= tol) { conv = true; break; }
        k_lm_precond<<<vg, 256, 0, st>>>(t, r, d, shift_S, n); h->n_launch++;
        if (m >= max_sub) {
            // restart from the current and the previous Ritz vectors; their
            // images are recomputed (near convergence the two are almost
            // parallel, and combining the old images would amplify rounding)
            ++restarts;
            double nu2;
            if ((rc = lm_dots(h, u, 1, u, &nu2, st))) return rc;
            k_axpby<<<vg, 256, 0, st>>>(1.0 / std::sqrt(nu2), u, 0.0, V, n);
            h->n_launch++;
            m = 1;
            if (have_prev) {
                double b, g2;
                if ((rc = lm_dots(h, V, 1, up, &b, st))) return rc;
                k_axpby<<<vg, 256, 0, st>>>(1.0, up, 0.0, V + ld, n);
                k_axpby<<<vg, 256, 0, st>>>(-b, V, 1.0, V + ld, n);
                h->n_launch += 2;
                if ((rc = lm_dots(h, V + ld, 1, V + ld, &g2, st))) return rc;
                if (g2 > 0.0 && std::isfinite(g2)) {
                    k_axpby<<<vg, 256, 0, st>>>(0.0, V + ld, 1.0 / std::sqrt(g2), V + ld, n);
                    h->n_launch++;
                    m = 2;
                }
            }
            for (int j = 0; j < m; ++j) {
                if ((rc = lm_apply(h, V + (size_t)j * ld, HV + (size_t)j * ld, SV + (size_t)j * ld, store, stream)))
                    return rc;
                k_axpby<<<vg, 256, 0, st>>>(shift_H, V + (size_t)j * ld + 1, 1.0, HV + (size_t)j * ld + 1, n - 1);
                k_axpby<<<vg, 256, 0, st>>>(shift_S, V + (size_t)j * ld + 1, 1.0, SV + (size_t)j * ld + 1, n - 1);
                h->n_launch += 2;
            }
            // the projected matrices of the kept columns
            for (int j = 0; j < m; ++j) {
                if ((rc = lm_dots(h, V, m, HV + (size_t)j * ld, col.data(), st))) return rc;
                if ((rc = lm_dots(h, HV, m, V + (size_t)j * ld, row.data(), st))) return rc;
                for (int i = 0; i < m; ++i) hm[(size_t)i * max_sub + j] = hm[(size_t)j * max_sub + i] = 0.5 * (col[i] + row[i]);
                if ((rc = lm_dots(h, V, m, SV + (size_t)j * ld, col.data(), st))) return rc;
                if ((rc = lm_dots(h, SV, m, V + (size_t)j * ld, row.data(), st))) return rc;
                for (int i = 0; i < m; ++i) sm[(size_t)i * max_sub + j] = sm[(size_t)j * max_sub + i] = 0.5 * (col[i] + row[i]);
            }
        }
        // keep the current Ritz vector as the previous one
        VCK(cudaMemcpyAsync(up, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        have_prev = true;
        VCK(launch_ok());
    }
    // x = u / u_0 and (S x)_0
    double u0, su0;
    VCK(cudaMemcpyAsync(&u0, u, sizeof(double), cudaMemcpyDeviceToHost, st));
    VCK(cudaMemcpyAsync(&su0, Su, sizeof(double), cudaMemcpyDeviceToHost, st));
    VCK(cudaStreamSynchronize(st));
    if (!(u0 != 0.0) || !std::isfinite(u0)) return VMC_ERR_NONFINITE;
    k_axpby<<<vg, 256, 0, st>>>(1.0 / u0, u, 0.0, x, n); h->n_launch++;
    VCK(cudaGetLastError());
    VCK(cudaStreamSynchronize(st));
    if (info) {
        info->iterations = std::min(iters, max_iter);
        info->restarts = restarts;
        info->converged = conv ? 1 : 0;
        info->eigenvalue = theta;
        info->rel_residual = relres;
        info->Sx0 = su0 / u0;
    }
    return conv ? VMC_OK : VMC_ERR_NOT_CONVERGED;
}

extern "C" int lm_update(vmc_handle h, const double* x, double Sx0, void* stream) {
    if (!h || !x || !std::isfinite(Sx0) || Sx0 == 0.0) return VMC_ERR_INVALID_ARG;
    if (!h->params_set) return VMC_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    UpdateArgs a{};
    a.C64 = h->d_C64; a.C32 = h->d_C32; a.invC64 = h->d_invC64; a.invC32 = h->d_invC32;
    a.F64 = h->d_F64; a.F32 = h->d_F32; a.pq_of = h->d_pq_of;
    a.ncp = h->ncp; a.npf = h->npf; a.M = h->M;
    a.status = h->d_status;
    k_lm_update<<<vgrid(h, 1), 256, 0, st>>>(a, x, 1.0 / Sx0); h->n_launch++;
    VCK(cudaGetLastError());
    h->obar_ok[0] = h->obar_ok[1] = h->obar_ok[2] = false;
    h->sorted_ok = h->g_ok = h->corr_ok = false;
    return read_status(h, st);
}

// ---------------------------------------------------------------------------
// measurement support
// ---------------------------------------------------------------------------
static int fold_records(vmc_ctx* h) {
    for (auto& r : h->recs) {
        VCK(cudaEventSynchronize(r.b));
        float ms = 0.f;
        VCK(cudaEventElapsedTime(&ms, r.a, r.b));
        h->acc_ms[r.kind] += ms;
        h->acc_bytes[r.kind] += r.bytes;
        h->acc_n[r.kind] += 1;
        h->ev_pool.push_back(r.a);
        h->ev_pool.push_back(r.b);
    }
    h->recs.clear();
    return VMC_OK;
}

extern "C" int vmc_profile(vmc_handle h, int enable) {
    if (!h) return VMC_ERR_INVALID_ARG;
    int rc = fold_records(h);
    if (rc) return rc;
    for (int k = 0; k < 4; ++k) { h->acc_ms[k] = 0; h->acc_bytes[k] = 0; h->acc_n[k] = 0; }
    h->n_launch = 0;
    h->prof = enable != 0;
    return VMC_OK;
}

extern "C" int vmc_profile_read(vmc_handle h, int store, int64_t* launches_all, int64_t* pass_launches,
                                double* pass_ms, double* pass_bytes) {
    if (!h || store < 0 || store > 3) return VMC_ERR_INVALID_ARG;
    int rc = fold_records(h);
    if (rc) return rc;
    if (launches_all) *launches_all = h->n_launch;
    if (pass_launches) *pass_launches = h->acc_n[store];
    if (pass_ms) *pass_ms = h->acc_ms[store];
    if (pass_bytes) *pass_bytes = h->acc_bytes[store];
    return VMC_OK;
}

// ---------------------------------------------------------------------------
// several problems in one streaming launch
// ---------------------------------------------------------------------------
extern "C" int sr_apply_S_batch(const vmc_handle* hs, int n, const double* const* V, double* const* out,
                                double shift, int store, void* stream) {
    if (!hs || !V || !out || n < 1 || n > kMaxBatch) return VMC_ERR_INVALID_ARG;
    if (store != VMC_STORE_FP64 && store != VMC_STORE_FP32) return VMC_ERR_INVALID_ARG;
    const int kind = store == VMC_STORE_FP64 ? 0 : 1;
    for (int b = 0; b < n; ++b) {
        if (!hs[b] || !V[b] || !out[b]) return VMC_ERR_INVALID_ARG;
        if (hs[b]->n_s == 0 || !store_ptr(hs[b], kind)) return VMC_ERR_STATE;
        if (hs[b]->dev != hs[0]->dev) return VMC_ERR_INVALID_ARG;
        for (int c = 0; c < b; ++c)
            if (hs[c] == hs[b]) return VMC_ERR_INVALID_ARG;
    }
    vmc_ctx* h0 = hs[0];
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<MainArgs<double>> args(n);
    std::vector<int> cta0(n + 1, 0);
    // CTAs in proportion to each problem's stored bytes, about two per SM in all
    size_t smem = 0;
    double work = 0.0;
    for (int b = 0; b < n; ++b) work += (double)hs[b]->n_s * (hs[b]->P + hs[b]->ncorr);
    for (int b = 0; b < n; ++b) {
        vmc_ctx* h = hs[b];
        int rc = ensure_obar(h, kind, st);
        if (rc) return rc;
        k_dot_part<double, double, 1><<<vgrid(h, 1), 256, 0, st>>>(h->d_Obar[kind], V[b], h->nv, h->part(0), nullptr);
        h->n_launch++;
        smem = std::max(smem, main_smem(h, 1, sizeof(double)));
        const double share = (double)h->n_s * (h->P + h->ncorr) / work;
        int g = (int)std::ceil(share * 2 * h0->nsm);
        g = (int)std::max<int64_t>(1, std::min<int64_t>(g, (h->n_s + 15) / 16));
        g = std::min<int64_t>(g, (int64_t)(h->pfpart_bytes / ((size_t)h->npf * sizeof(double))));
        cta0[b + 1] = cta0[b] + g;
        MainArgs<double>& a = args[b];
        a.pb = h->pb;
        a.n_s = h->n_s;
        a.s_occ = h->d_socc; a.Nst = h->Nst;
        a.s_cidx = h->d_cidx; a.ncst = h->ncst;
        a.s_pf = store_ptr(h, kind); a.Pst = h->Pst;
        a.V = V[b]; a.invC = h->d_invC64; a.T = (double*)h->d_T;
        a.pf_partial = (double*)h->d_pfpart;
        a.stop = nullptr;
    }
    if (smem > h0->smem_optin) { set_err("pairing block does not fit in shared memory"); return VMC_ERR_UNSUPPORTED; }
    void* dbuf = nullptr;
    const size_t abytes = round_up(sizeof(MainArgs<double>) * n, 256);
    int rc = batch_buffer(h0, abytes + sizeof(int) * (n + 1), &dbuf);
    if (rc) return rc;
    MainArgs<double>* dargs = (MainArgs<double>*)dbuf;
    int* dcta = (int*)((unsigned char*)dbuf + abytes);
    VCK(cudaMemcpyAsync(dargs, args.data(), sizeof(MainArgs<double>) * n, cudaMemcpyHostToDevice, st));
    VCK(cudaMemcpyAsync(dcta, cta0.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
    VCK(launch_sr_main_batch(kind == 0 ? 8 : 4, cta0[n], smem, st, dargs, dcta, n));
    h0->n_launch++;
    for (int b = 0; b < n; ++b) {
        vmc_ctx* h = hs[b];
        if ((rc = launch_corr<double, 1>(h, (double*)h->d_T, nullptr, st))) return rc;
        if ((rc = reduce_pf<double>(h, cta0[b + 1] - cta0[b], 1, st))) return rc;
        FinArgs<double, double> f{};
        f.pb = h->pb;
        f.n_s = h->n_s;
        f.inv_n = 1.0 / (double)h->n_s;
        f.centered = 0;
        f.pf_partial = (const double*)h->d_pfpart;
        f.pf_raw = h->d_pfraw;
        f.corr_raw = h->d_corrraw;
        f.invC = h->d_invC64;
        f.ObarA = h->d_Obar[kind];
        f.obv_part = h->part(0);
        f.n_obv_part = vgrid(h, 1);
        f.V = V[b];
        f.shift = shift;
        f.out = out[b];
        f.dot_part = nullptr;
        f.stop = nullptr;
        k_finalize_S<double, double, 1><<<vgrid(h, 1), 256, 0, st>>>(f); h->n_launch++;
        VCK(cudaGetLastError());
    }
    // the host copies of the argument blocks must outlive the launch's copies
    VCK(cudaStreamSynchronize(st));
    return VMC_OK;
}

