// Fused single-pass Eq. 7 product over the sorted BF16 rows G (one vector).
//
// (S v)_k needs, per sample s, t_s = O_s . v and then sum_s t_s O_s.  G holds
// every pairing element of a sample as (pq << 16) | bf16, in kGParts parts of
// consecutive pq, each in a bank-aware order (k_build_G in sorted.cu, once per
// set of samples), so the index work is paid once per SR step and both halves
// of the product run in one pass:
//
//   * a group of kGParts warps takes one sample at a time; warp f of the group
//     holds part f of the sample's G row in registers and loads its part of
//     the next row while it works on the current one (bulk prefetches bring
//     the rows after that into L2);
//   * gather: each warp sums W_e v[pq_e] over its part (v in one shared-memory
//     table per CTA) and a share of the correlator terms v_k / C_k; the
//     group's partial sums meet in shared memory behind one named barrier;
//   * scatter: each warp adds (t_s - Obar . v) W_e for its part to the
//     group's own shared-memory image of the pairing block.  The image
//     belongs to one group, the group works on one sample at a time and its
//     parts cover disjoint pq, so the update is a plain load, add and store
//     (shared-memory atomics cost about five plain accesses on this GPU).
//
// kFusedImages images of 8,128 floats plus the v table fill 227 KB at 56
// electrons / 128 spin orbitals, so an SM runs 6 groups of 4 warps.  The
// images are summed per CTA at the end; k_sv_finish sums the CTAs and runs
// the correlator half of the transposed product from the correlator runs.
// The parameter-major copy T of the two-pass product is not read: each
// product streams G (4 bytes per element) once.
#include "common.cuh"
#include "kernels.h"
#include "corr_runs.cuh"

namespace vmc {

__device__ __forceinline__ void group_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int U>
__global__ void __launch_bounds__(kFusedWarps * 32, 1) k_sv_fused(SortedArgs a, float* pf_partial, int wq) {
    if (a.stop && *a.stop) return;
    constexpr int F = kGParts, NI = kFusedImages, NW = kFusedWarps;
    extern __shared__ __align__(16) unsigned char smem[];
    const DevProblem& pb = a.pb;
    const int npf = pb.npf, ncorr = pb.ncorr;
    const float* __restrict__ vpf = (const float*)smem;
    float* img = (float*)smem + npf;                         // [NI][npf]
    int* coff = (int*)(img + (size_t)NI * npf);
    __shared__ float part[NI][2][F];
    __shared__ float obv_s;
    __shared__ double red[NW];
    for (int i = threadIdx.x; i < npf; i += blockDim.x) ((float*)smem)[i] = a.V[pb.ncp + i];
    for (int i = threadIdx.x; i < NI * npf; i += blockDim.x) img[i] = 0.f;
    for (int i = threadIdx.x; i <= ncorr; i += blockDim.x) coff[i] = (int)pb.corr_off[i];
    if (threadIdx.x < 32) {
        const double c = warp_sum_partials(a.obv_part, a.n_obv_part, 0, 1);
        if (threadIdx.x == 0) obv_s = (float)c;
    }
    __syncthreads();
    const float obv = obv_s;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int gi = wid / F, f = wid % F;
    float* my = img + (size_t)gi * npf;
    // this warp's correlators: [c0, c1)
    const int cpf = (ncorr + F - 1) / F;
    const int c0 = min(ncorr, f * cpf), c1 = min(ncorr, c0 + cpf);
    const int64_t woff = (int64_t)f * wq;                   // first 16-byte word of this part
    const uint32_t part_bytes = (uint32_t)wq * 16;
    double tt = 0.0;
    const int64_t gstride = (int64_t)gridDim.x * NI;
    const int64_t s_first = (int64_t)blockIdx.x * NI + gi;
    // rows kFusedAhead samples ahead are requested into L2 by bulk prefetches,
    // which hold no registers or shared memory
    if (lane == 0)
        for (int d = 1; d <= kFusedAhead; ++d)
            if (s_first + d * gstride < a.n_s) prefetch_l2((const uint4*)(a.G + (s_first + d * gstride) * a.Pst) + woff,
                                                           part_bytes);
    uint4 g[U];
    {
        const uint4* g4 = (const uint4*)(a.G + s_first * a.Pst) + woff;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = lane + 32 * u;
            g[u] = (s_first < a.n_s && i < wq) ? __ldcs(g4 + i) : make_uint4(0u, 0u, 0u, 0u);
        }
    }
    int par = 0;
    for (int64_t s = s_first; s < a.n_s; s += gstride, par ^= 1) {
        if (lane == 0 && s + (kFusedAhead + 1) * gstride < a.n_s)
            prefetch_l2((const uint4*)(a.G + (s + (kFusedAhead + 1) * gstride) * a.Pst) + woff, part_bytes);
        uint4 gn[U];
        {
            const int64_t sn = s + gstride;
            const uint4* g4n = (const uint4*)(a.G + sn * a.Pst) + woff;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = lane + 32 * u;
                gn[u] = (sn < a.n_s && i < wq) ? __ldcs(g4n + i) : make_uint4(0u, 0u, 0u, 0u);
            }
        }
        // correlator terms v_k / C_k of this warp's share (issued before the
        // pairing loop, added after it)
        float cv = 0.f;
        {
            const cstate_t* cid = a.s_cidx + s * a.ncst;
            for (int c = c0 + lane; c < c1; c += 32) {
                const int k = coff[c] + (int)cid[c];
                cv += __ldg(a.V + k) * __ldg(a.invC + k);
            }
        }
        float t = 0.f, w = 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t e[4] = {g[u].x, g[u].y, g[u].z, g[u].w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float x = __uint_as_float(e[j] << 16) * vpf[e[j] >> 16];
                if (j & 1) w += x;
                else t += x;
            }
        }
        const float tw = warp_sum(t + w + cv);
        if (lane == 0) part[gi][par][f] = tw;
        group_barrier(1 + gi, 32 * F);
        float ts = 0.f;
#pragma unroll
        for (int k = 0; k < F; ++k) ts += part[gi][par][k];
        const float tc = ts - obv;
        if (f == 0 && lane == 0) {
            a.Tv[s] = tc;
            tt += (double)tc * tc;
        }
        // the group's parts cover disjoint pq, and the pq of one part are
        // distinct, so the image entries of up to 8 elements are loaded
        // together before any is written back; padding slots and exact zeros
        // are (0, 0.0) and skipped, so a padding lane never races with the
        // element of pq 0 in the same instruction
#pragma unroll
        for (int u0 = 0; u0 < U; u0 += 2) {
            float o[8];
#pragma unroll
            for (int u = u0; u < u0 + 2 && u < U; ++u) {
                const uint32_t e[4] = {g[u].x, g[u].y, g[u].z, g[u].w};
#pragma unroll
                for (int j = 0; j < 4; ++j) o[4 * (u - u0) + j] = (e[j] & 0xFFFFu) ? my[e[j] >> 16] : 0.f;
            }
#pragma unroll
            for (int u = u0; u < u0 + 2 && u < U; ++u) {
                const uint32_t e[4] = {g[u].x, g[u].y, g[u].z, g[u].w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (e[j] & 0xFFFFu) my[e[j] >> 16] = fmaf(tc, __uint_as_float(e[j] << 16), o[4 * (u - u0) + j]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) g[u] = gn[u];
    }
    if (lane == 0) red[wid] = tt;
    __syncthreads();
    float* dst = pf_partial + (size_t)blockIdx.x * npf;
    for (int i = threadIdx.x; i < npf; i += blockDim.x) {
        float x = 0.f;
#pragma unroll
        for (int k = 0; k < NI; ++k) x += img[(size_t)k * npf + i];
        dst[i] = x;
    }
    if (threadIdx.x == 0 && a.tt_part) {
        double v = 0.0;
        for (int k = 0; k < NW; ++k) v += red[k];
        a.tt_part[blockIdx.x] = v;
    }
}

// Correlator half of the transposed product (CTAs [0, nhist): shared-memory
// histograms of (class, sample slice); or, for classes too large for shared
// memory, CTAs [0, ncb): 8 work items of the correlator runs each) and the sum
// of the per-CTA pairing images (the other CTAs, one pairing amplitude per
// thread, CTAs in a fixed order).
__global__ void __launch_bounds__(256) k_sv_finish(SortedArgs a, const float* pf_partial, int nblk) {
    if (a.stop && *a.stop) return;
    extern __shared__ __align__(16) unsigned char hist_smem[];
    __shared__ float slots[8][32];
    int b = (int)blockIdx.x;
    if (b < a.nhist) {
        corr_hist_cta<1>(a, b / a.hist_slices, b % a.hist_slices, a.hist_slices, (float*)hist_smem);
        return;
    }
    b -= a.nhist;
    if (b < a.ncb) {
        const int64_t i = (int64_t)b * 8 + (threadIdx.x >> 5);
        if (i < (int64_t)*a.n_items) scatter_C_item<1>(a, a.items[i], slots[threadIdx.x >> 5]);
        return;
    }
    const int pq = (b - a.ncb) * blockDim.x + threadIdx.x;
    if (pq >= a.pb.npf) return;
    const int npf = a.pb.npf;
    // 16 independent loads in flight per thread, summed in a fixed order
    float s = 0.f;
    for (int c0 = 0; c0 < nblk; c0 += 16) {
        float x[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) x[c] = c0 + c < nblk ? pf_partial[(size_t)(c0 + c) * npf + pq] : 0.f;
#pragma unroll
        for (int c = 0; c < 16; ++c) s += x[c];
    }
    a.raw[pq] = s;
}

template __global__ void k_sv_fused<1>(SortedArgs, float*, int);
template __global__ void k_sv_fused<2>(SortedArgs, float*, int);
template __global__ void k_sv_fused<3>(SortedArgs, float*, int);
template __global__ void k_sv_fused<4>(SortedArgs, float*, int);

}  // namespace vmc
