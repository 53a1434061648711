// Correlator half of the transposed product from the correlator runs: the
// samples of every correlator parameter grouped by parameter (built once per
// set of samples, see sorted.cu), summed against the per-sample dots t_s.
#pragma once
#include "common.cuh"
#include "kernels.h"

namespace vmc {

// Correlator part of the gather for one sample: lane L looks up V[k_c] / C[k_c]
// for c = L + 32 j (at most 32 kCorrPerLane correlators).  The loads are only
// issued here; the caller adds cv after its pairing work, which hides them.
template <int K>
__device__ __forceinline__ void corr_lookups(const DevProblem& pb, const int* coff, const cstate_t* cid,
                                             const float* V, const float* invC, int lane,
                                             float (&cv)[kCorrPerLane][K]) {
#pragma unroll
    for (int j = 0; j < kCorrPerLane; ++j) {
        const int c = lane + 32 * j;
#pragma unroll
        for (int kk = 0; kk < K; ++kk) cv[j][kk] = 0.f;
        if (c < pb.ncorr) {
            const int k = coff[c] + (int)cid[c];
            const float ic = __ldg(invC + k);
#pragma unroll
            for (int kk = 0; kk < K; ++kk) cv[j][kk] = __ldg(V + kk * pb.nv + k) * ic;
        }
    }
}

// dst[0..K) += x[0..K) in global memory, one (vector) reduction
template <int K>
__device__ __forceinline__ void red_add(float* dst, const float (&x)[K]) {
    if constexpr (K == 4) {
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(x[0]), "f"(x[1]), "f"(x[2]),
                     "f"(x[3])
                     : "memory");
    } else if constexpr (K == 2) {
        asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(dst), "f"(x[0]), "f"(x[1]) : "memory");
    } else {
        atomicAdd(dst, x[0]);
    }
}

// Correlator half of the transposed product as a weighted histogram: CTA
// (class q, slice j) adds the centered t_s of its slice of the samples at
// the state of every correlator of class q into a shared-memory histogram of
// the class's 4^m amplitudes, then adds each nonzero bin to craw (one global
// vector reduction per bin and slice).  The states are read correlator-major
// (coalesced), t_s sample-major.
template <int K>
__device__ __forceinline__ void corr_hist_cta(const SortedArgs& a, int q, int j, int nsl, float* hist) {
    const DevProblem& pb = a.pb;
    const int64_t off = pb.class_off[q];
    const int d = (int)(pb.class_off[q + 1] - off);
    // hist[kk][state]: the bins of one component spread over all banks
    for (int i = threadIdx.x; i < d * K; i += blockDim.x) hist[i] = 0.f;
    __syncthreads();
    const int64_t per = (a.n_s + nsl - 1) / nsl;
    const int64_t s0 = min(a.n_s, (int64_t)j * per), s1 = min(a.n_s, s0 + per);
    const int bd = blockDim.x;
    for (int ci = pb.class_ptr[q]; ci < pb.class_ptr[q + 1]; ++ci) {
        const cstate_t* st = a.cidxT + (int64_t)pb.class_inst[ci] * a.n_s;
        int64_t s = s0 + threadIdx.x;
        // four samples per thread in flight: the loads first, then the adds
        for (; s + 3 * bd < s1; s += 4 * bd) {
            int k[4];
            float t[4][K];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                k[u] = (int)st[s + u * bd];
#pragma unroll
                for (int kk = 0; kk < K; ++kk) t[u][kk] = a.Tv[(s + u * bd) * K + kk];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int kk = 0; kk < K; ++kk) atomicAdd(&hist[kk * d + k[u]], t[u][kk]);
        }
        for (; s < s1; s += bd) {
            const int k = (int)st[s];
#pragma unroll
            for (int kk = 0; kk < K; ++kk) atomicAdd(&hist[kk * d + k], a.Tv[s * K + kk]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        float x[K];
        bool nz = false;
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            x[kk] = hist[kk * d + i];
            nz |= x[kk] != 0.f;
        }
        if (nz) red_add<K>(a.craw + (off + i) * K, x);
    }
}

// Correlator work item (group g, entries e0 .. min(e0 + kCorrItem, end of g)):
// the group's parameters 32 g .. 32 g + 31 have contiguous runs, read as one
// coalesced stream; entries carry k mod 32, equal values are contiguous, and
// a segmented warp scan hands each segment's sum to its last lane, which adds
// it to the parameter's slot in shared memory (one writer per parameter per
// step).  The slots are then added to craw (zeroed by the caller): a long run
// (a parameter shared by many correlators) spreads over several items.
template <int K>
__device__ __forceinline__ void scatter_C_item(const SortedArgs& a, uint2 item, float* slot) {
    const int lane = threadIdx.x & 31;
    const int64_t k0 = (int64_t)item.x * 32;
    const int64_t kend = min(a.pb.ncp, k0 + 32);
#pragma unroll
    for (int kk = 0; kk < K; ++kk) slot[lane * K + kk] = 0.f;
    __syncwarp();
    const uint32_t lo = item.y, hi = min(a.cbase[kend], lo + (uint32_t)kCorrItem);
    for (uint32_t e0 = lo; e0 < hi; e0 += 32) {
        const uint32_t e = e0 + lane;
        const bool in = e < hi;
        const uint32_t v = in ? __ldcs(a.Tc + e) : 0u;
        const int ls = in ? (int)(v & 31u) : 32 + lane;        // past the end: a segment of its own
        float t[K];
#pragma unroll
        for (int kk = 0; kk < K; ++kk) t[kk] = in ? __ldg(a.Tv + (int64_t)(v >> 5) * K + kk) : 0.f;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int lo_ls = __shfl_up_sync(0xffffffffu, ls, o);
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                const float u = __shfl_up_sync(0xffffffffu, t[kk], o);
                if (lane >= o && lo_ls == ls) t[kk] += u;
            }
        }
        const int next_ls = __shfl_down_sync(0xffffffffu, ls, 1);
        if (in && (lane == 31 || next_ls != ls))
#pragma unroll
            for (int kk = 0; kk < K; ++kk) slot[ls * K + kk] += t[kk];
        __syncwarp();
    }
    if (k0 + lane < kend)
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const float v = slot[lane * K + kk];
            if (v != 0.f) atomicAdd(a.craw + (k0 + lane) * K + kk, v);
        }
}

}  // namespace vmc
