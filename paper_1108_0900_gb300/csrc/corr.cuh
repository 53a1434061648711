// Correlator half of the Eq. 7 product on a thread-block cluster, shared by
// the stand-alone correlator kernel and the fused scatter kernel.
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace vmc {

// The kCorrCluster CTAs of the cluster for work unit u (a class q and up to
// kInstPerUnit of its correlators, which share the class's parameter block)
// histogram t_s over the 4^m states, each CTA for a slice of the samples, into
// their own shared memory h (4^m x K values of AT); after a cluster barrier
// CTA r sums its share of the states over the cluster's histograms through
// distributed shared memory (fixed order) and adds them to
// corr_raw[class_off_q + state] (zeroed by the caller; a class with more
// correlators spreads over several units).
// Slices start on multiples of 8 samples; each thread takes 8 consecutive
// samples per step (two 16-byte loads of states, K x 8 values of t).  Every
// CTA of the cluster must call this.
template <typename AT, int K>
__device__ __forceinline__ void corr_cluster_histogram(const CorrArgs<AT>& a, AT* h, int u) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const DevProblem& pb = a.pb;
    const int rank = (int)cluster.block_rank();
    const int4 unit = a.units[u];                 // class, correlators [y, z) of class_inst
    const int q = unit.x;
    const int64_t off = pb.class_off[q];
    const int d = (int)(pb.class_off[q + 1] - off);
    for (int i = threadIdx.x; i < d * K; i += blockDim.x) h[i] = AT(0);
    __syncthreads();
    const int64_t len = ((a.n_s + kCorrCluster - 1) / kCorrCluster + 7) & ~(int64_t)7;
    const int64_t s0 = min(a.n_s, rank * len), s1 = min(a.n_s, s0 + len);
    // 16-byte loads need the rows to start on a 16-byte boundary
    const bool vec = ((a.n_s & 7) == 0);
    for (int ji = unit.y; ji < unit.z; ++ji) {
        const cstate_t* st = a.cidxT + (int64_t)pb.class_inst[ji] * a.n_s;
        int64_t s = s0;
        if (vec) {
            for (int64_t g = s0 + 8 * (int64_t)threadIdx.x; g + 8 <= s1; g += 8 * (int64_t)blockDim.x) {
                const uint4 sa = *(const uint4*)(st + g), sb = *(const uint4*)(st + g + 4);
                const uint32_t w8[8] = {sa.x, sa.y, sa.z, sa.w, sb.x, sb.y, sb.z, sb.w};
                AT tv[8 * K];
#pragma unroll
                for (int j = 0; j < 8 * K; ++j) tv[j] = a.T[g * K + j];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int i = (int)w8[j];
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) atomicAdd(&h[i * K + kk], tv[j * K + kk]);
                }
            }
            s = s0 + ((s1 - s0) & ~(int64_t)7);
        }
        for (int64_t qs = s + threadIdx.x; qs < s1; qs += blockDim.x) {
            int i = st[qs];
#pragma unroll
            for (int kk = 0; kk < K; ++kk) atomicAdd(&h[i * K + kk], a.T[qs * K + kk]);
        }
    }
    cluster.sync();
    const int per = (d + kCorrCluster - 1) / kCorrCluster;
    const int b0 = min(d, rank * per) * K, b1 = min(d, (rank + 1) * per) * K;
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
        double acc = 0.0;
#pragma unroll
        for (int r = 0; r < kCorrCluster; ++r) acc += (double)cluster.map_shared_rank(h, r)[i];
        if (acc != 0.0) atomicAdd(a.corr_raw + off * K + i, (AT)acc);   // several units may share a class
    }
    cluster.sync();   // keep this CTA's histogram alive until the cluster has read it
}

}  // namespace vmc
