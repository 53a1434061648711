// SR kernels over the stored derivative ratios (Sec. II.A):
//   - the matrix-free product of Eq. 7, (1/n_s) sum_s O_s (O_s . v), with the
//     covariance term -Obar (Obar . v) and the absolute shift eps v;
//   - the sample means Obar, <E_L> and the gradient g = <E_L O> - <E_L> Obar;
//   - the vector updates of conjugate gradient with FP64 scalars.
//
// Per sample the O vector is sparse: correlator c contributes 1/C at its own
// parameter off_c + idx_c, and the pairing block holds P values W_e on the
// pairs of occupied orbitals.  A pass therefore streams the O store once:
//   gather   t_s = sum_c v[k_c]/C[k_c] + sum_e W_e v[pq(e)],
//   scatter  out[pq(e)] += t_s W_e into a per-CTA shared-memory image of the
//            pairing block (written out as one partial per CTA),
// and the correlator scatter runs correlator-major over a transposed state
// array into shared-memory histograms of each correlator's 4^m states, one
// per CTA of a thread-block cluster, summed through distributed shared
// memory, so neither half uses global atomics.
#include <cooperative_groups.h>
#include <type_traits>
#include "common.cuh"
#include "corr.cuh"
#include "kernels.h"

namespace vmc {

template <typename ST, typename AT> __device__ __forceinline__ AT load_st(const void* p, int64_t i);
template <> __device__ __forceinline__ double load_st<double, double>(const void* p, int64_t i) {
    return __ldg((const double*)p + i);
}
template <> __device__ __forceinline__ double load_st<float, double>(const void* p, int64_t i) {
    return (double)__ldg((const float*)p + i);
}
template <> __device__ __forceinline__ float load_st<float, float>(const void* p, int64_t i) {
    return __ldg((const float*)p + i);
}
template <> __device__ __forceinline__ float load_st<__nv_bfloat16, float>(const void* p, int64_t i) {
    return __bfloat162float(((const __nv_bfloat16*)p)[i]);
}
template <> __device__ __forceinline__ double load_st<__nv_bfloat16, double>(const void* p, int64_t i) {
    return (double)__bfloat162float(((const __nv_bfloat16*)p)[i]);
}

// FP32 store with FP64-accurate sums in FP32 arithmetic.  The FP64 pipe of
// this GPU retires one warp FMA per 16 cycles per SM, and the FP64 form of
// this pass (conversions, FMAs and FP64 shared atomics) is bound by it.
// Here the v table holds each FP64 value as an FP32 pair (hi, lo); a product
// w v = w hi + w lo is split exactly into its rounded value and the FMA error
// term; the per-lane sums are FP32 pairs kept by Knuth's two-sum; the image
// of the pairing block is two FP32 arrays: the first atomic add returns the
// old value, so the rounding error of the add it made is known exactly and
// is added to the second array with the product's error terms.  The rounded
// intrinsics keep the compiler from fusing the error arithmetic.
__device__ __forceinline__ void ff_add(float& sh, float& sl, float p, float err) {
    const float s = __fadd_rn(sh, p);
    const float bp = __fsub_rn(s, sh);
    const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(e, err));
}

template <int K, bool GATHER>
__device__ void sr_main_run_ff(const MainArgs<double>& a, int cta, int ncta, unsigned char* smem) {
    const DevProblem& pb = a.pb;
    const int npf = pb.npf, M = pb.M, N = pb.N, P = pb.P;
    float* hi = (float*)smem;                    // [npf][K] image, rounded sums
    float* lo = hi + (size_t)npf * K;            // [npf][K] their rounding errors
    float2* vpf = (float2*)(lo + (size_t)npf * K);
    int* rowbase = (int*)(vpf + (GATHER ? (size_t)npf * K : 0));
    uint8_t* occw = (uint8_t*)(rowbase + M);
    for (int i = threadIdx.x; i < 2 * npf * K; i += blockDim.x) hi[i] = 0.f;
    if (GATHER)
        for (int i = threadIdx.x; i < npf; i += blockDim.x)
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const double v = a.V[kk * pb.nv + pb.ncp + i];
                const float vh = (float)v;
                vpf[i * K + kk] = make_float2(vh, (float)(v - (double)vh));
            }
    for (int i = threadIdx.x; i < M; i += blockDim.x) rowbase[i] = pb.rowbase[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint8_t* my = occw + wid * 64;
    const float* pf = (const float*)a.s_pf;
    for (int64_t s = (int64_t)cta * nw + wid; s < a.n_s; s += (int64_t)ncta * nw) {
        for (int i = lane; i < N; i += 32) my[i] = a.s_occ[s * a.Nst + i];
        __syncwarp();
        double t[K];
        if (GATHER) {
            double tc[K];
            float sh[K], sl[K];
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                tc[kk] = 0.0;
                sh[kk] = sl[kk] = 0.f;
            }
            for (int c = lane; c < pb.ncorr; c += 32) {
                const int64_t k = pb.corr_off[c] + a.s_cidx[s * a.ncst + c];
                const double ic = a.invC[k];
#pragma unroll
                for (int kk = 0; kk < K; ++kk) tc[kk] += a.V[kk * pb.nv + k] * ic;
            }
            // four elements per lane in flight: the loads first
            for (int e0 = lane; e0 < P; e0 += 128) {
                int pq[4];
                float w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + 32 * u;
                    w[u] = e < P ? __ldg(pf + s * a.Pst + e) : 0.f;
                    const uint16_t pt = e < P ? pb.pairtab[e] : (uint16_t)0;
                    pq[u] = rowbase[my[pt & 255]] + my[pt >> 8];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (e0 + 32 * u >= P) continue;
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        const float2 v = vpf[pq[u] * K + kk];
                        const float p = __fmul_rn(w[u], v.x);
                        ff_add(sh[kk], sl[kk], p, __fadd_rn(fmaf(w[u], v.x, -p), __fmul_rn(w[u], v.y)));
                    }
                }
            }
#pragma unroll
            for (int kk = 0; kk < K; ++kk) t[kk] = warp_sum((double)sh[kk] + (double)sl[kk] + tc[kk]);
            if (lane < K) {
                double mine = t[0];
#pragma unroll
                for (int kk = 1; kk < K; ++kk) if (lane == kk) mine = t[kk];
                a.T[s * K + lane] = mine;
            }
        } else {
#pragma unroll
            for (int kk = 0; kk < K; ++kk) t[kk] = a.T[s * K + kk];
        }
        float th[K], tl[K];
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            th[kk] = (float)t[kk];
            tl[kk] = (float)(t[kk] - (double)th[kk]);
        }
        for (int e0 = lane; e0 < P; e0 += 128) {
            int pq[4];
            float w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = e0 + 32 * u;
                w[u] = e < P ? __ldg(pf + s * a.Pst + e) : 0.f;
                const uint16_t pt = e < P ? pb.pairtab[e] : (uint16_t)0;
                pq[u] = rowbase[my[pt & 255]] + my[pt >> 8];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (e0 + 32 * u >= P) continue;
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    const float p = __fmul_rn(th[kk], w[u]);
                    const float err = __fadd_rn(fmaf(th[kk], w[u], -p), __fmul_rn(tl[kk], w[u]));
                    const float old = atomicAdd(&hi[pq[u] * K + kk], p);
                    const float sum = __fadd_rn(old, p);
                    const float bp = __fsub_rn(sum, old);
                    const float e2 = __fadd_rn(__fsub_rn(old, __fsub_rn(sum, bp)), __fsub_rn(p, bp));
                    atomicAdd(&lo[pq[u] * K + kk], __fadd_rn(e2, err));
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();
    double* dst = a.pf_partial + (size_t)cta * npf * K;
    for (int i = threadIdx.x; i < npf * K; i += blockDim.x) dst[i] = (double)hi[i] + (double)lo[i];
}

// The generic pass for one problem, run by CTA `cta` of `ncta` serving it.
template <typename ST, typename AT, int K, bool GATHER>
__device__ void sr_main_run(const MainArgs<AT>& a, int cta, int ncta, unsigned char* smem) {
    if constexpr (std::is_same<ST, float>::value && std::is_same<AT, double>::value) {
        if (a.pb.ff_sums) {
            sr_main_run_ff<K, GATHER>(a, cta, ncta, smem);
            return;
        }
    }
    const DevProblem& pb = a.pb;
    const int npf = pb.npf, M = pb.M, N = pb.N, P = pb.P;
    AT* acc = (AT*)smem;
    AT* vpf = acc + (size_t)npf * K;
    int* rowbase = (int*)(vpf + (GATHER ? (size_t)npf * K : 0));
    uint8_t* occw = (uint8_t*)(rowbase + M);
    for (int i = threadIdx.x; i < npf * K; i += blockDim.x) acc[i] = AT(0);
    if (GATHER)
        for (int i = threadIdx.x; i < npf; i += blockDim.x)
#pragma unroll
            for (int kk = 0; kk < K; ++kk) vpf[i * K + kk] = a.V[kk * pb.nv + pb.ncp + i];
    for (int i = threadIdx.x; i < M; i += blockDim.x) rowbase[i] = pb.rowbase[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint8_t* my = occw + wid * 64;
    for (int64_t s = (int64_t)cta * nw + wid; s < a.n_s; s += (int64_t)ncta * nw) {
        for (int i = lane; i < N; i += 32) my[i] = a.s_occ[s * a.Nst + i];
        __syncwarp();
        AT t[K];
        if (GATHER) {
#pragma unroll
            for (int kk = 0; kk < K; ++kk) t[kk] = AT(0);
            for (int c = lane; c < pb.ncorr; c += 32) {
                int64_t k = pb.corr_off[c] + a.s_cidx[s * a.ncst + c];
                AT ic = a.invC[k];
#pragma unroll
                for (int kk = 0; kk < K; ++kk) t[kk] += a.V[kk * pb.nv + k] * ic;
            }
            for (int e = lane; e < P; e += 32) {
                uint16_t pt = pb.pairtab[e];
                int pq = rowbase[my[pt & 255]] + my[pt >> 8];
                AT w = load_st<ST, AT>(a.s_pf, s * a.Pst + e);
#pragma unroll
                for (int kk = 0; kk < K; ++kk) t[kk] += w * vpf[pq * K + kk];
            }
#pragma unroll
            for (int kk = 0; kk < K; ++kk) t[kk] = warp_sum(t[kk]);
            if (lane < K) {
                AT mine = t[0];
#pragma unroll
                for (int kk = 1; kk < K; ++kk) if (lane == kk) mine = t[kk];
                a.T[s * K + lane] = mine;
            }
        } else {
#pragma unroll
            for (int kk = 0; kk < K; ++kk) t[kk] = a.T[s * K + kk];
        }
        for (int e = lane; e < P; e += 32) {
            uint16_t pt = pb.pairtab[e];
            int pq = rowbase[my[pt & 255]] + my[pt >> 8];
            AT w = load_st<ST, AT>(a.s_pf, s * a.Pst + e);
#pragma unroll
            for (int kk = 0; kk < K; ++kk) atomicAdd(&acc[pq * K + kk], t[kk] * w);
        }
        __syncwarp();
    }
    __syncthreads();
    AT* dst = a.pf_partial + (size_t)cta * npf * K;
    for (int i = threadIdx.x; i < npf * K; i += blockDim.x) dst[i] = acc[i];
}

template <typename ST, typename AT, int K, bool GATHER>
__global__ void __launch_bounds__(512) k_sr_main(MainArgs<AT> a) {
    if (a.stop && *a.stop) return;
    extern __shared__ __align__(16) unsigned char smem[];
    sr_main_run<ST, AT, K, GATHER>(a, blockIdx.x, gridDim.x, smem);
}

// Several problems in one launch: CTAs [cta0[b], cta0[b + 1]) serve problem
// b, each with the shared-memory layout of its own problem.
template <typename ST, typename AT>
__global__ void __launch_bounds__(512) k_sr_main_batch(const MainArgs<AT>* __restrict__ args,
                                                       const int* __restrict__ cta0, int n) {
    extern __shared__ __align__(16) unsigned char smem[];
    int b = 0;
    while (b + 1 < n && (int)blockIdx.x >= cta0[b + 1]) ++b;
    if ((int)blockIdx.x >= cta0[n]) return;
    sr_main_run<ST, AT, 1, true>(args[b], blockIdx.x - cta0[b], cta0[b + 1] - cta0[b], smem);
}

// correlator scatter for classes of more states than shared memory holds:
// every (correlator, sample) adds t_s to its parameter in global memory
template <typename AT, int K>
__global__ void __launch_bounds__(256) k_corr_scatter_global(CorrArgs<AT> a) {
    if (a.stop && *a.stop) return;
    const DevProblem& pb = a.pb;
    const int c = blockIdx.y;
    const cstate_t* st = a.cidxT + (int64_t)c * a.n_s;
    const int64_t off = pb.corr_off[c];
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.n_s; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = off + st[s];
#pragma unroll
        for (int kk = 0; kk < K; ++kk) atomicAdd(a.corr_raw + k * K + kk, a.T[s * K + kk]);
    }
}

// correlator-major scatter: one thread-block cluster per correlator class
template <typename AT, int K>
__global__ void __cluster_dims__(kCorrCluster, 1, 1) __launch_bounds__(256) k_corr_scatter(CorrArgs<AT> a) {
    if (a.stop && *a.stop) return;   // uniform over the grid: no CTA reaches a cluster barrier
    extern __shared__ __align__(16) unsigned char smem[];
    corr_cluster_histogram<AT, K>(a, (AT*)smem, blockIdx.x / kCorrCluster);
}

template <int K>
__device__ __forceinline__ void block_reduce_store(double (&v)[K], double* out) {
    __shared__ double red[K][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        double x = warp_sum(v[kk]);
        if (lane == 0) red[kk][wid] = x;
    }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            double x = lane < nw ? red[kk][lane] : 0.0;
            x = warp_sum(x);
            if (lane == 0) out[blockIdx.x * K + kk] = x;
        }
    }
}

// Reduce the per-CTA pairing-block images: raw[pq][kk] = sum_b part[b][pq][kk].
// Block = 32 parameter slots x 8 CTA slices; a warp covers one slice.
template <typename AT>
__global__ void __launch_bounds__(256) k_reduce_pf(const AT* part, int nblk, int npfK, AT* raw) {
    __shared__ double red[8][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (i < npfK)
        for (int b = w; b < nblk; b += 8) s += (double)part[(int64_t)b * npfK + i];
    red[w][lane] = s;
    __syncthreads();
    if (w == 0) {
        double t = 0.0;
#pragma unroll
        for (int j = 0; j < 8; ++j) t += red[j][lane];
        if (i < npfK) raw[i] = (AT)t;
    }
}

// raw pass result for parameter k and vector kk, divided by n_s (in AT)
template <typename AT, typename VT, int K>
__device__ __forceinline__ AT fin_raw(const FinArgs<AT, VT>& a, int64_t k, int kk) {
    const DevProblem& pb = a.pb;
    const AT raw = k < pb.ncp ? a.corr_raw[k * K + kk] * a.invC[k] : a.pf_raw[(k - pb.ncp) * K + kk];
    return raw * (AT)a.inv_n;
}

// Vector kernels cover kVecUnroll elements per thread, strided by the grid,
// with every load of the body issued before the arithmetic: one launch over
// the 270k-parameter vectors is one round trip to memory per thread.
constexpr int kVecUnroll = 4;

// out = raw - Obar (Obar . V) + shift V; dot_part = partial out . V.  A
// centered pass (t_s - Obar . V scattered) already holds the covariance and
// skips the Obar term.  Element arithmetic in AT, partial dots in FP64.
template <typename AT, typename VT, int K>
__global__ void __launch_bounds__(256) k_finalize_S(FinArgs<AT, VT> a) {
    if (a.stop && *a.stop) return;
    __shared__ double obv[K];
    if (threadIdx.x < 32) {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            double s = a.centered ? 0.0 : warp_sum_partials(a.obv_part, a.n_obv_part, kk, K);
            if (threadIdx.x == 0) obv[kk] = s;
        }
    }
    __syncthreads();
    AT ov[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) ov[kk] = (AT)obv[kk];
    const AT shift = (AT)a.shift;
    const int64_t nv = a.pb.nv;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double dl[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) dl[kk] = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < nv; i0 += kVecUnroll * stride) {
        AT ob[kVecUnroll], v[kVecUnroll][K], raw[kVecUnroll][K];
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t k = i0 + u * stride;
            ob[u] = AT(0);
#pragma unroll
            for (int kk = 0; kk < K; ++kk) v[u][kk] = raw[u][kk] = AT(0);
            if (k < nv) {
                if (!a.centered) ob[u] = a.ObarA[k];
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    v[u][kk] = (AT)a.V[kk * nv + k];
                    raw[u][kk] = fin_raw<AT, VT, K>(a, k, kk);
                }
            }
        }
        AT part[K];
#pragma unroll
        for (int kk = 0; kk < K; ++kk) part[kk] = AT(0);
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t k = i0 + u * stride;
            if (k < nv) {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    const AT o = raw[u][kk] - ob[u] * ov[kk] + shift * v[u][kk];
                    a.out[kk * nv + k] = (VT)o;
                    part[kk] += o * v[u][kk];
                }
            }
        }
#pragma unroll
        for (int kk = 0; kk < K; ++kk) dl[kk] += (double)part[kk];
    }
    if (a.dot_part) block_reduce_store<K>(dl, a.dot_part);
}

// gradient mode: K = 2 with t_s = (1, E_s)
template <typename AT>
__global__ void __launch_bounds__(256) k_finalize_grad(FinArgs<AT, double> a) {
    __shared__ double em;
    if (threadIdx.x < 32) {
        double s = warp_sum_partials(a.E_sum, a.n_E_part, 0, 1);
        if (threadIdx.x == 0) em = s * a.inv_n;
    }
    __syncthreads();
    const int64_t nv = a.pb.nv;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nv; k += (int64_t)gridDim.x * blockDim.x) {
        double o = fin_raw<AT, double, 2>(a, k, 0);
        double eo = fin_raw<AT, double, 2>(a, k, 1);
        a.Obar_out[k] = o;
        a.g_out[k] = eo - em * o;
    }
}

// ---------------------------------------------------------------------------
// small vector kernels
// ---------------------------------------------------------------------------
__global__ void k_build_T_grad(const double* E, int64_t n_s, double* T, double* E_part) {
    double loc[1] = {0.0};
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_s; s += (int64_t)gridDim.x * blockDim.x) {
        T[2 * s] = 1.0;
        T[2 * s + 1] = E[s];
        loc[0] += E[s];
    }
    block_reduce_store<1>(loc, E_part);
}

// partial dots: part[blk][kk] = sum_i a[i] b[kk n + i]
template <typename TA, typename TB, int K>
__global__ void __launch_bounds__(256) k_dot_part(const TA* x, const TB* y, int64_t n, double* part, const int* stop) {
    if (stop && *stop) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double loc[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) loc[kk] = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVecUnroll * stride) {
        double xv[kVecUnroll], yv[kVecUnroll][K];
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t i = i0 + u * stride;
            xv[u] = i < n ? (double)x[i] : 0.0;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) yv[u][kk] = i < n ? (double)y[kk * n + i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u)
#pragma unroll
            for (int kk = 0; kk < K; ++kk) loc[kk] += xv[u] * yv[u][kk];
    }
    block_reduce_store<K>(loc, part);
}

__global__ void k_transpose_cidx(const cstate_t* cidx, int ncst, int ncorr, int64_t n_s, cstate_t* cidxT) {
    // tile 32 samples x 32 correlators
    __shared__ cstate_t tile[32][33];
    int64_t s0 = (int64_t)blockIdx.x * 32;
    int c0 = blockIdx.y * 32;
    int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        int64_t s = s0 + r;
        int c = c0 + tx;
        tile[r][tx] = (s < n_s && c < ncorr) ? cidx[s * ncst + c] : 0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        int c = c0 + r;
        int64_t s = s0 + tx;
        if (c < ncorr && s < n_s) cidxT[(int64_t)c * n_s + s] = tile[tx][r];
    }
}

template <typename VT>
__global__ void k_cast(const double* src, VT* dst, int64_t n, double scale) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (VT)(src[i] * scale);
}

// ---------------------------------------------------------------------------
// conjugate gradient on (S + eps I) x = b, FP64 scalars in `scal`:
//   scal[0] rr, scal[1] |b|^2, scal[2] tol^2, scal[3] iterations, scal[4] rr_prev
// ---------------------------------------------------------------------------

__device__ __forceinline__ double sum_part(const double* part, int n, int kk, int K) {
    double s = 0.0;
    for (int b = 0; b < n; ++b) s += part[b * K + kk];
    return s;
}

template <typename VT>
__global__ void __launch_bounds__(256) k_cg_init(const VT* b, VT* x, VT* r, VT* p, int64_t n, double* part) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double loc[1] = {0.0};
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVecUnroll * stride) {
        VT bv[kVecUnroll];
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t i = i0 + u * stride;
            bv[u] = i < n ? b[i] : VT(0);
        }
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                x[i] = VT(0);
                r[i] = bv[u];
                p[i] = bv[u];
                loc[0] += (double)bv[u] * (double)bv[u];
            }
        }
    }
    block_reduce_store<1>(loc, part);
}

__global__ void k_cg_start(const double* part, int npart, double* scal, double tol, int* stop) {
    double rr = warp_sum_partials(part, npart, 0, 1);
    if (threadIdx.x != 0) return;
    scal[CG_RR] = rr;
    scal[CG_BB] = rr;
    scal[CG_TOL2] = tol * tol * rr;
    scal[CG_IT] = 0.0;
    scal[CG_RRP] = rr;
    *stop = (rr == 0.0) ? 1 : 0;
}

// alpha = rr / (p . Ap); x += alpha p; r -= alpha Ap; partial r . r
// (element arithmetic in VT, partial sums in FP64)
template <typename VT>
__global__ void __launch_bounds__(256) k_cg_xr(VT* x, VT* r, const VT* p, const VT* Ap, int64_t n,
                                               const double* pAp_part, int npart, double* scal,
                                               double* rr_part, int* stop) {
    if (*stop) return;
    __shared__ double alpha;
    if (threadIdx.x < 32) {
        double pAp = warp_sum_partials(pAp_part, npart, 0, 1);
        if (threadIdx.x == 0) {
            alpha = scal[CG_RR] / pAp;
            if (!isfinite(alpha) || pAp <= 0.0) alpha = 0.0;
        }
    }
    __syncthreads();
    const VT al = (VT)alpha;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double loc[1] = {0.0};
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVecUnroll * stride) {
        VT xv[kVecUnroll], rv[kVecUnroll], pv[kVecUnroll], qv[kVecUnroll];
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t i = i0 + u * stride;
            const bool in = i < n;
            xv[u] = in ? x[i] : VT(0);
            rv[u] = in ? r[i] : VT(0);
            pv[u] = in ? p[i] : VT(0);
            qv[u] = in ? Ap[i] : VT(0);
        }
        VT part = VT(0);
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                const VT xi = xv[u] + al * pv[u];
                const VT ri = rv[u] - al * qv[u];
                x[i] = xi;
                r[i] = ri;
                part += ri * ri;
            }
        }
        loc[0] += (double)part;
    }
    block_reduce_store<1>(loc, rr_part);
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[CG_RRP] = scal[CG_RR];
}

// two block sums to two partial arrays
__device__ __forceinline__ void block_reduce_store2(double a, double b, double* out_a, double* out_b) {
    __shared__ double red[2][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) { red[0][wid] = a; red[1][wid] = b; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        double x = lane < nw ? red[0][lane] : 0.0, y = lane < nw ? red[1][lane] : 0.0;
        x = warp_sum(x);
        y = warp_sum(y);
        if (lane == 0) { out_a[blockIdx.x] = x; out_b[blockIdx.x] = y; }
    }
}

// Fused CG update after a centered product.  With t_s - Obar . p scattered,
// the curvature is p . (S + eps) p = (1/n) sum_s (t_s - Obar . p)^2 + eps |p|^2,
// both known from partial sums (gather, previous p update), so alpha needs no
// separate dot product and Ap = raw / n + eps p is formed element by element
// and never stored: x += alpha p; r -= alpha Ap; partial r . r.
template <typename VT>
__device__ __forceinline__ void cg_fxr_body(const CgFusedArgs<VT>& a) {
    __shared__ double alpha;
    if (threadIdx.x < 32) {
        const double tt = warp_sum_partials(a.tt_part, a.ntt, 0, 1);
        const double pp = warp_sum_partials(a.pp_part, a.npp, 0, 1);
        if (threadIdx.x == 0) {
            const double pAp = tt * a.inv_n + a.shift * pp;
            alpha = a.scal[CG_RR] / pAp;
            if (!isfinite(alpha) || pAp <= 0.0) alpha = 0.0;
        }
    }
    __syncthreads();
    const VT al = (VT)alpha, inv_n = (VT)a.inv_n, sh = (VT)a.shift;
    const int64_t n = a.n, stride = (int64_t)gridDim.x * blockDim.x;
    double loc[1] = {0.0};
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVecUnroll * stride) {
        VT xv[kVecUnroll], rv[kVecUnroll], pv[kVecUnroll], raw[kVecUnroll];
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t i = i0 + u * stride;
            const bool in = i < n;
            xv[u] = in ? a.x[i] : VT(0);
            rv[u] = in ? a.r[i] : VT(0);
            pv[u] = in ? a.p[i] : VT(0);
            raw[u] = !in ? VT(0) : i < a.ncp ? a.corr_raw[i] * a.invC[i] : a.pf_raw[i - a.ncp];
            if (in && i < a.ncp) a.corr_raw[i] = VT(0);   // ready for the next product's additions
        }
        VT part = VT(0);
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                const VT q = raw[u] * inv_n + sh * pv[u];
                const VT ri = rv[u] - al * q;
                a.x[i] = xv[u] + al * pv[u];
                a.r[i] = ri;
                part += ri * ri;
            }
        }
        loc[0] += (double)part;
    }
    block_reduce_store<1>(loc, a.rr_part);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.scal[CG_RRP] = a.scal[CG_RR];
}

template <typename VT>
__global__ void __launch_bounds__(256) k_cg_fxr(CgFusedArgs<VT> a) {
    if (*a.stop) return;
    cg_fxr_body(a);
}

// beta = rr_new / rr; p = r + beta p; partials Obar . p (centering of the next
// product) and |p|^2 (its curvature)
template <typename VT>
__device__ __forceinline__ void cg_p_body(const VT* r, VT* p, int64_t n, const double* rr_part, int npart,
                                          double* scal, const VT* Obar, double* obp_part, double* pp_part,
                                          int* stop, int max_iter) {
    __shared__ double beta, rrn;
    if (threadIdx.x < 32) {
        double r = warp_sum_partials(rr_part, npart, 0, 1);
        if (threadIdx.x == 0) {
            rrn = r;
            beta = rrn / scal[CG_RRP];
        }
    }
    __syncthreads();
    const VT be = (VT)beta;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double lo = 0.0, lp = 0.0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kVecUnroll * stride) {
        VT rv[kVecUnroll], pv[kVecUnroll], ov[kVecUnroll];
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t i = i0 + u * stride;
            const bool in = i < n;
            rv[u] = in ? r[i] : VT(0);
            pv[u] = in ? p[i] : VT(0);
            ov[u] = in ? Obar[i] : VT(0);
        }
        VT po = VT(0), pp = VT(0);
#pragma unroll
        for (int u = 0; u < kVecUnroll; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                const VT pi = rv[u] + be * pv[u];
                p[i] = pi;
                po += ov[u] * pi;
                pp += pi * pi;
            }
        }
        lo += (double)po;
        lp += (double)pp;
    }
    block_reduce_store2(lo, lp, obp_part, pp_part);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        scal[CG_RR] = rrn;
        double it = scal[CG_IT] + 1.0;
        scal[CG_IT] = it;
        if (rrn <= scal[CG_TOL2] || !isfinite(rrn) || it >= (double)max_iter) *stop = 1;
    }
}

template <typename VT>
__global__ void __launch_bounds__(256) k_cg_p(const VT* r, VT* p, int64_t n, const double* rr_part, int npart,
                                              double* scal, const VT* Obar, double* obp_part, double* pp_part,
                                              int* stop, int max_iter) {
    if (*stop) return;
    cg_p_body(r, p, n, rr_part, npart, scal, Obar, obp_part, pp_part, stop, max_iter);
}

// Both CG updates in one cooperative launch: x/r (with the r . r partials),
// a grid-wide barrier, then beta and p (with the partials of the next
// product); saves a launch and its start-up per inner iteration.  The grid
// must be co-resident (cudaLaunchCooperativeKernel checks it).
template <typename VT>
__global__ void __launch_bounds__(256) k_cg_fxrp(CgFusedArgs<VT> a, const VT* Obar, double* obp_part,
                                                 int* stop, int max_iter) {
    if (*a.stop) return;
    cg_fxr_body(a);
    cooperative_groups::this_grid().sync();
    cg_p_body<VT>(a.r, const_cast<VT*>(a.p), a.n, a.rr_part, (int)gridDim.x, a.scal, Obar, obp_part,
                  const_cast<double*>(a.pp_part), stop, max_iter);
}

// The same two updates when the grid covers the vectors in one pass (each
// thread owns elements i0 + u * stride, u < kVecUnroll): the thread loads x,
// r, p, the product and Obar once, before the partial sums that give alpha
// are reduced, and keeps r and p in registers across the grid barrier, so
// the p update reads nothing from memory.  Same arithmetic, element by
// element and in every partial sum, as k_cg_fxrp.
template <typename VT>
__global__ void __launch_bounds__(256) k_cg_fxrp1(CgFusedArgs<VT> a, const VT* Obar, double* obp_part,
                                                  int* stop, int max_iter) {
    if (*a.stop) return;
    const int64_t n = a.n, stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    VT xv[kVecUnroll], rv[kVecUnroll], pv[kVecUnroll], raw[kVecUnroll], ov[kVecUnroll];
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
        const int64_t i = i0 + u * stride;
        const bool in = i < n;
        xv[u] = in ? a.x[i] : VT(0);
        rv[u] = in ? a.r[i] : VT(0);
        pv[u] = in ? a.p[i] : VT(0);
        raw[u] = !in ? VT(0) : i < a.ncp ? a.corr_raw[i] * a.invC[i] : a.pf_raw[i - a.ncp];
        ov[u] = in ? Obar[i] : VT(0);
        if (in && i < a.ncp) a.corr_raw[i] = VT(0);   // ready for the next product's additions
    }
    __shared__ double alpha, beta, rrn;
    if (threadIdx.x < 32) {
        const double tt = warp_sum_partials(a.tt_part, a.ntt, 0, 1);
        const double pp = warp_sum_partials(a.pp_part, a.npp, 0, 1);
        if (threadIdx.x == 0) {
            const double pAp = tt * a.inv_n + a.shift * pp;
            alpha = a.scal[CG_RR] / pAp;
            if (!isfinite(alpha) || pAp <= 0.0) alpha = 0.0;
        }
    }
    __syncthreads();
    const VT al = (VT)alpha, inv_n = (VT)a.inv_n, sh = (VT)a.shift;
    VT part = VT(0);
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
        const int64_t i = i0 + u * stride;
        if (i < n) {
            const VT q = raw[u] * inv_n + sh * pv[u];
            const VT ri = rv[u] - al * q;
            a.x[i] = xv[u] + al * pv[u];
            a.r[i] = ri;
            rv[u] = ri;
            part += ri * ri;
        }
    }
    double loc[1] = {(double)part};
    block_reduce_store<1>(loc, a.rr_part);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.scal[CG_RRP] = a.scal[CG_RR];
    cooperative_groups::this_grid().sync();
    if (threadIdx.x < 32) {
        const double r2 = warp_sum_partials(a.rr_part, (int)gridDim.x, 0, 1);
        if (threadIdx.x == 0) {
            rrn = r2;
            beta = r2 / a.scal[CG_RRP];
        }
    }
    __syncthreads();
    const VT be = (VT)beta;
    VT po = VT(0), pp = VT(0);
#pragma unroll
    for (int u = 0; u < kVecUnroll; ++u) {
        const int64_t i = i0 + u * stride;
        if (i < n) {
            const VT pi = rv[u] + be * pv[u];
            const_cast<VT*>(a.p)[i] = pi;
            po += ov[u] * pi;
            pp += pi * pi;
        }
    }
    block_reduce_store2((double)po, (double)pp, obp_part, const_cast<double*>(a.pp_part));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.scal[CG_RR] = rrn;
        const double it = a.scal[CG_IT] + 1.0;
        a.scal[CG_IT] = it;
        if (rrn <= a.scal[CG_TOL2] || !isfinite(rrn) || it >= (double)max_iter) *stop = 1;
    }
}

// partial sums of x (FP64)
__global__ void __launch_bounds__(256) k_vec_sum(const double* x, int64_t n, double* part) {
    double loc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        loc[0] += x[i];
    block_reduce_store<1>(loc, part);
}

// SR parameter update (Sec. II.A, after Eq. 2).  x_0 = 1 - tau <E_L> + tau Obar . y
// from the partial sums (every block forms the same value), then alpha_k +=
// -tau y_k / x_0 with the derived copies: C in FP32, 1/C in both precisions,
// and both triangles of the antisymmetric F.  A non-positive or non-finite
// x_0 changes nothing and sets ST_NONFINITE.
__global__ void __launch_bounds__(256) k_sr_update(UpdateArgs a) {
    __shared__ double x0s;
    if (threadIdx.x < 32) {
        const double e = warp_sum_partials(a.e_part, a.ne, 0, 1) * a.inv_n;
        const double oy = warp_sum_partials(a.oy_part, a.noy, 0, 1);
        if (threadIdx.x == 0) x0s = 1.0 - a.tau * e + a.tau * oy;
    }
    __syncthreads();
    const double x0 = x0s;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.x0 = x0;
    if (!(x0 > 0.0) || !isfinite(x0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.status, ST_NONFINITE);
        return;
    }
    const double s = -a.tau / x0;
    const int64_t nv = a.ncp + a.npf;
    int bad = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nv; k += (int64_t)gridDim.x * blockDim.x) {
        const double d = s * a.y[k];
        if (k < a.ncp) {
            const double c = a.C64[k] + d;
            if (c == 0.0) bad |= ST_SINGULAR;
            if (!isfinite(c)) bad |= ST_NONFINITE;
            a.C64[k] = c;
            a.C32[k] = (float)c;
            a.invC64[k] = 1.0 / c;
            a.invC32[k] = (float)(1.0 / c);
        } else {
            const uint32_t pq = a.pq_of[k - a.ncp];
            const int p = (int)(pq & 0xFFFFu), q = (int)(pq >> 16);
            const double f = a.F64[(int64_t)p * a.M + q] + d;
            if (!isfinite(f)) bad |= ST_NONFINITE;
            a.F64[(int64_t)p * a.M + q] = f;
            a.F64[(int64_t)q * a.M + p] = -f;
            a.F32[(int64_t)p * a.M + q] = (float)f;
            a.F32[(int64_t)q * a.M + p] = -(float)f;
        }
    }
    if (bad) atomicOr(a.status, bad);
}

// out = n (out + Obar (Obar . v)): undo the covariance term of a product
// formed with shift 0, leaving the plain sum_s (O_s . v) O_s
__global__ void __launch_bounds__(256) k_uncenter(double* out, const double* Obar, const double* obv_part, int nobv,
                                                  double n_s, int64_t nv) {
    __shared__ double obv;
    if (threadIdx.x < 32) {
        const double s = warp_sum_partials(obv_part, nobv, 0, 1);
        if (threadIdx.x == 0) obv = s;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = n_s * (out[i] + Obar[i] * obv);
}

// y = a - b (FP64)
__global__ void k_sub(const double* a, const double* b, double* y, int64_t n, double* part) {
    double loc[1] = {0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = a[i] - b[i];
        y[i] = v;
        loc[0] += v * v;
    }
    block_reduce_store<1>(loc, part);
}

// y = a x + b y (FP64)
__global__ void k_axpby(double a, const double* x, double b, double* y, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = b == 0.0 ? a * x[i] : a * x[i] + b * y[i];   // b = 0: y may hold anything
}

// x64 += scale * d
template <typename VT>
__global__ void k_axpy_to64(double* x, const VT* d, double scale, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += scale * (double)d[i];
}

// ---------------------------------------------------------------------------
// explicit instantiations used by the host side
// ---------------------------------------------------------------------------
template __global__ void k_sr_main<double, double, 1, true>(MainArgs<double>);

template __global__ void k_sr_main<double, double, 2, true>(MainArgs<double>);
template __global__ void k_sr_main<double, double, 4, true>(MainArgs<double>);
template __global__ void k_sr_main<double, double, 2, false>(MainArgs<double>);
template __global__ void k_sr_main<float, double, 1, true>(MainArgs<double>);
template __global__ void k_sr_main<float, double, 2, true>(MainArgs<double>);
template __global__ void k_sr_main<float, double, 4, true>(MainArgs<double>);
template __global__ void k_sr_main<float, double, 2, false>(MainArgs<double>);
template __global__ void k_sr_main<float, float, 1, true>(MainArgs<float>);
template __global__ void k_sr_main<float, float, 2, true>(MainArgs<float>);
template __global__ void k_sr_main<float, float, 4, true>(MainArgs<float>);
template __global__ void k_sr_main<__nv_bfloat16, double, 2, false>(MainArgs<double>);
template __global__ void k_sr_main<__nv_bfloat16, float, 1, true>(MainArgs<float>);
template __global__ void k_sr_main<__nv_bfloat16, float, 2, true>(MainArgs<float>);
template __global__ void k_sr_main<__nv_bfloat16, float, 4, true>(MainArgs<float>);
template __global__ void k_corr_scatter_global<double, 1>(CorrArgs<double>);
template __global__ void k_corr_scatter_global<double, 2>(CorrArgs<double>);
template __global__ void k_corr_scatter_global<double, 4>(CorrArgs<double>);
template __global__ void k_corr_scatter_global<float, 1>(CorrArgs<float>);
template __global__ void k_corr_scatter_global<float, 2>(CorrArgs<float>);
template __global__ void k_corr_scatter_global<float, 4>(CorrArgs<float>);
template __global__ void k_corr_scatter<double, 1>(CorrArgs<double>);
template __global__ void k_corr_scatter<double, 2>(CorrArgs<double>);
template __global__ void k_corr_scatter<double, 4>(CorrArgs<double>);
template __global__ void k_corr_scatter<float, 1>(CorrArgs<float>);
template __global__ void k_corr_scatter<float, 2>(CorrArgs<float>);
template __global__ void k_corr_scatter<float, 4>(CorrArgs<float>);
template __global__ void k_finalize_S<double, double, 1>(FinArgs<double, double>);
template __global__ void k_finalize_S<double, double, 2>(FinArgs<double, double>);
template __global__ void k_finalize_S<double, double, 4>(FinArgs<double, double>);
template __global__ void k_finalize_S<float, float, 1>(FinArgs<float, float>);
template __global__ void k_finalize_S<float, float, 2>(FinArgs<float, float>);
template __global__ void k_finalize_S<float, float, 4>(FinArgs<float, float>);
template __global__ void k_finalize_grad<double>(FinArgs<double, double>);
template __global__ void k_reduce_pf<double>(const double*, int, int, double*);
template __global__ void k_reduce_pf<float>(const float*, int, int, float*);
template __global__ void k_dot_part<double, double, 1>(const double*, const double*, int64_t, double*, const int*);
template __global__ void k_dot_part<double, double, 2>(const double*, const double*, int64_t, double*, const int*);
template __global__ void k_dot_part<double, double, 4>(const double*, const double*, int64_t, double*, const int*);
template __global__ void k_dot_part<double, float, 1>(const double*, const float*, int64_t, double*, const int*);
template __global__ void k_dot_part<double, float, 2>(const double*, const float*, int64_t, double*, const int*);
template __global__ void k_dot_part<double, float, 4>(const double*, const float*, int64_t, double*, const int*);
template __global__ void k_cast<float>(const double*, float*, int64_t, double);
template __global__ void k_cast<double>(const double*, double*, int64_t, double);
template __global__ void k_cg_init<double>(const double*, double*, double*, double*, int64_t, double*);
template __global__ void k_cg_init<float>(const float*, float*, float*, float*, int64_t, double*);
template __global__ void k_cg_xr<double>(double*, double*, const double*, const double*, int64_t, const double*, int,
                                         double*, double*, int*);
template __global__ void k_cg_xr<float>(float*, float*, const float*, const float*, int64_t, const double*, int,
                                        double*, double*, int*);
template __global__ void k_cg_p<double>(const double*, double*, int64_t, const double*, int, double*, const double*,
                                        double*, double*, int*, int);
template __global__ void k_cg_p<float>(const float*, float*, int64_t, const double*, int, double*, const float*,
                                       double*, double*, int*, int);
template __global__ void k_cg_fxr<float>(CgFusedArgs<float>);
template __global__ void k_cg_fxrp<float>(CgFusedArgs<float>, const float*, double*, int*, int);
template __global__ void k_cg_fxrp1<float>(CgFusedArgs<float>, const float*, double*, int*, int);
template __global__ void k_axpy_to64<float>(double*, const float*, double, int64_t);
template __global__ void k_axpy_to64<double>(double*, const double*, double, int64_t);


// launch of the batched generic pass from the unit that defines it (store_bytes
// 8: FP64 store, 4: FP32 store; FP64 accumulation)
cudaError_t launch_sr_main_batch(int store_bytes, int blocks, size_t smem, cudaStream_t st,
                                 const MainArgs<double>* args, const int* cta0, int n) {
    cudaError_t e;
    if (store_bytes == 8) {
        e = cudaFuncSetAttribute(k_sr_main_batch<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        k_sr_main_batch<double, double><<<blocks, 512, smem, st>>>(args, cta0, n);
    } else {
        e = cudaFuncSetAttribute(k_sr_main_batch<float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        k_sr_main_batch<float, double><<<blocks, 512, smem, st>>>(args, cta0, n);
    }
    return cudaGetLastError();
}

}  // namespace vmc
