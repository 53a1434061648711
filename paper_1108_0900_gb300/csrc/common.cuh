// Device-side helpers shared by the vmcsr kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define VMC_FULL_MASK 0xffffffffu

namespace vmc {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11), written from the published rounds:
// two 32x32->64 multiplies per round with multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

__host__ __device__ inline u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        u32x4 n;
        n.x = (uint32_t)(p1 >> 32) ^ c.y ^ k0;
        n.y = (uint32_t)p1;
        n.z = (uint32_t)(p0 >> 32) ^ c.w ^ k1;
        n.w = (uint32_t)p0;
        c = n;
    }
    return c;
}

// ---------------------------------------------------------------------------
// warp reductions
// ---------------------------------------------------------------------------
// request [p, p + bytes) into L2 (16-byte aligned, a multiple of 16 bytes);
// holds no registers or shared memory while the data is on its way
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(VMC_FULL_MASK, v, o);
    return v;
}
template <typename T> __device__ __forceinline__ T warp_prod(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(VMC_FULL_MASK, v, o);
    return v;
}

// n-th (0-based) set bit of a 64-bit mask; caller guarantees popc(mask) > n
__device__ __forceinline__ int nth_set_bit64(uint64_t mask, int n) {
    uint32_t lo = (uint32_t)mask, hi = (uint32_t)(mask >> 32);
    int cl = __popc(lo);
    if (n < cl) return __fns(lo, 0, n + 1);
    return 32 + __fns(hi, 0, n - cl + 1);
}

__device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
}

template <typename R> struct real_traits;
template <> struct real_traits<float> {
    static __device__ __forceinline__ float from_bf16(__nv_bfloat16 x) { return __bfloat162float(x); }
};
template <> struct real_traits<double> {};

// status bits written by kernels (host reads them after a sync)
enum StatusBits : int {
    ST_SINGULAR = 1,
    ST_NONFINITE = 2,
    ST_BAD_CONFIG = 4,
    ST_TIMEOUT = 8,
};

// ---------------------------------------------------------------------------
// Device view of a problem.  All arrays are device pointers owned by the
// handle.
// ---------------------------------------------------------------------------
// correlator state index sum_j 4^j (n_up + 2 n_dn) of one correlator (up to
// 9 sites: 18 bits)
using cstate_t = uint32_t;

struct DevProblem {
    int ns;        // spatial orbitals
    int M;         // spin orbitals
    int nu, nd, N; // electrons
    int ncorr;
    int P;         // pairing block per sample = nu(nu-1)/2 + nd(nd-1)/2 + nu nd
    int npf;       // M(M-1)/2
    int ham;       // 0 Hubbard, 1 ab initio
    int64_t ncp;   // correlator parameters
    int64_t nv;    // all parameters
    double U;
    // correlators
    const int* corr_ptr;       // [ncorr+1]
    const int* corr_sites;     // flattened site lists
    const int64_t* corr_off;   // [ncorr+1] first parameter of each correlator's block, then ncp
    int max_csites;            // sites of the largest correlator
    int ff_sums;               // FP32-store passes with FP64 sums: FP32-pair arithmetic instead of FP64
    int n_class;               // parameter classes (correlators of a class share a block)
    const int64_t* class_off;  // [n_class+1] parameter blocks of the classes
    const int* class_ptr;      // [n_class+1] into class_inst
    const int* class_inst;     // correlators grouped by class
    // site -> (correlator, 4^j) memberships
    const int* site_cptr;      // [ns+1]
    const int* site_corr;      // correlator id
    const int* site_w;         // 4^j weight of the site inside that correlator
    const uint32_t* corr_site_w;   // [ncorr][ns] 4^j weight of site s in correlator c, 0 if absent
    // Hubbard hopping lists: site s hops to nbr_site[k] with amplitude nbr_t[k]
    const int* nbr_ptr;        // [ns+1]
    const int* nbr_site;
    const double* nbr_t;
    // ab initio integrals (spatial indices): h[ns][ns], eri[((p ns + q) ns + r) ns + s] = (pq|rs)
    const double* h64;
    const float* h32;
    const double* eri64;
    const float* eri32;
    // correlators containing both sites i and j: pair_corr[pair_ptr[i ns + j] ..]
    const int* pair_ptr;
    const int* pair_corr;
    int pair_unique;           // no site pair lies in two correlators (and ncp < 2^30): per-sample pair table
    // double excitations: electron-position pairs (a | b << 8) of the up-up,
    // down-down and up-down classes, then empty-orbital index pairs (ix | iy << 8)
    // of the same classes (ab initio only)
    const uint16_t* dexc;
    // parameters
    const double* C64;
    const float* C32;
    const double* F64;         // M x M antisymmetric
    const float* F32;
    // pairing block decoding: e -> (a | b << 8) over ascending positions
    const uint16_t* pairtab;   // [P]
    const int* rowbase;        // [M]: f_pq index = rowbase[p] + q (p < q)
};

// sum of n partials (stride K, column kk) by one warp; all lanes get it.
// Eight loads per lane are issued before they are added (fixed order), so up
// to 256 partials cost one round trip to L2.
__device__ __forceinline__ double warp_sum_partials(const double* part, int n, int kk, int K) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b0 = 0; b0 < n; b0 += 256) {
        double v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int b = b0 + lane + 32 * j;
            v[j] = b < n ? part[b * K + kk] : 0.0;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) s += v[j];
    }
    return warp_sum(s);
}

__host__ __device__ inline int64_t pf_row_base(int M, int p) {
    // index(p, q) = p M - p (p + 1) / 2 + (q - p - 1) = base(p) + q
    return (int64_t)p * M - (int64_t)p * (p + 1) / 2 - p - 1;
}

}  // namespace vmc
