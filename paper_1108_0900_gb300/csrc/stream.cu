// TMA-staged streaming pass over the O store: the matrix-free product of
// Eq. 7, t_s = O_s . v followed by sum_s t_s O_s, for the low-precision stores
// (BF16 or FP32 storage, FP32 accumulation).
//
// Staging.  Every warp owns two shared-memory buffers and one mbarrier per
// buffer.  Lane 0 fetches a sample's record (ascending occupation,
// correlator states, pairing block) with three 1-D bulk copies
// (cp.async.bulk, complete_tx on the buffer's mbarrier) two samples ahead,
// so each warp keeps ~2 records in flight while it computes on a third.
// Every wait is bounded: a wait that runs out sets ST_TIMEOUT and the warp
// drains its own copies (bounded again) before it stops.
//
// Pairing block.  With positions 0..nu-1 spin up and nu..N-1 spin down, the
// block holds the up-up and down-down triangles and the up-down rectangle.
// Lane l owns column l of a block; the orbital of every position sits in a
// register (ou = up orbital l, od = down orbital l) and rows are fetched by
// shuffles, so an element costs one shared load of W, one gather of v and
// one atomic add.  The two triangles are walked two rows at a time (row i
// together with row nu-2-i) so all nu lanes stay busy.  Along a row the
// parameter index is base(p) + q with q ascending inside one spin block, so
// a warp touches a window of <= 64 consecutive words: at most 2-way bank
// conflicts for the gather and the scatter.
#include "common.cuh"
#include "kernels.h"

namespace vmc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: true when the phase completed
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < (1u << 22); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <typename ST> __device__ __forceinline__ float ld_w(const ST* w, int i);
template <> __device__ __forceinline__ float ld_w<float>(const float* w, int i) { return w[i]; }
template <> __device__ __forceinline__ float ld_w<__nv_bfloat16>(const __nv_bfloat16* w, int i) {
    return __bfloat162float(w[i]);
}

__device__ __forceinline__ int rowbase_of(int p, int M) { return ((p * (2 * M - 3 - p)) >> 1) - 1; }

// One pass over a record for one triangle (spin block with n electrons whose
// ascending orbitals are in register `o` of lanes 0..n-1, block offset off).
// PHASE 0 gathers into t, PHASE 1 scatters t into acc.
template <typename ST, int K, int PHASE>
__device__ __forceinline__ void tri_block(const ST* W, int off, int n, int o, int M, const float* vpf, float* acc,
                                          float (&t)[K]) {
    const int lane = threadIdx.x & 31;
    const int iters = n / 2;  // rows 0..n-2 paired as (i, n-2-i); n-1 rows in all
    for (int i = 0; i < iters; ++i) {
        const int r1 = i, r2 = n - 2 - i;
        int r, b;
        bool valid = lane < n;
        if (lane > r1) { r = r1; b = lane; }
        else { r = r2; b = r2 + 1 + lane; valid = valid && (r1 < r2); }
        if (b >= n) { valid = false; b = 0; }
        const int p = __shfl_sync(VMC_FULL_MASK, o, r);
        const int q = __shfl_sync(VMC_FULL_MASK, o, b);
        if (valid) {
            const int pq = rowbase_of(p, M) + q;
            const int e = off + r * n - ((r * (r + 1)) >> 1) + (b - r - 1);
            const float w = ld_w<ST>(W, e);
            if (PHASE == 0) {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) t[kk] += w * vpf[pq * K + kk];
            } else {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) atomicAdd(&acc[pq * K + kk], t[kk] * w);
            }
        }
    }
}

template <typename ST, int K, int PHASE>
__device__ __forceinline__ void rect_block(const ST* W, int off, int nu, int nd, int ou, int od, int M,
                                           const float* vpf, float* acc, float (&t)[K]) {
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < nu; ++r) {
        const int p = __shfl_sync(VMC_FULL_MASK, ou, r);
        if (lane < nd) {
            const int pq = rowbase_of(p, M) + od;
            const float w = ld_w<ST>(W, off + r * nd + lane);
            if (PHASE == 0) {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) t[kk] += w * vpf[pq * K + kk];
            } else {
#pragma unroll
                for (int kk = 0; kk < K; ++kk) atomicAdd(&acc[pq * K + kk], t[kk] * w);
            }
        }
    }
}

template <typename ST, int K>
__global__ void __launch_bounds__(512, 1) k_sr_stream(StreamArgs a) {
    if (a.stop && *a.stop) return;
    extern __shared__ __align__(128) unsigned char smem[];
    const DevProblem& pb = a.pb;
    const int npf = pb.npf, M = pb.M, nu = pb.nu, nd = pb.nd;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // layout: acc | vpf | corr offsets | mbarriers | staging buffers
    float* acc = (float*)smem;
    float* vpf = acc + (size_t)npf * K;
    int* coff = (int*)(vpf + (size_t)npf * K);
    uint64_t* bars = (uint64_t*)(smem + (((size_t)npf * K * 8 + (size_t)(pb.ncorr + 1) * 4 + 15) & ~(size_t)15));
    unsigned char* bufs = (unsigned char*)(bars + 2 * nw);
    bufs = (unsigned char*)(((uintptr_t)bufs + 127) & ~(uintptr_t)127);

    for (int i = threadIdx.x; i < npf * K; i += blockDim.x) acc[i] = 0.f;
    for (int i = threadIdx.x; i < npf; i += blockDim.x)
#pragma unroll
        for (int kk = 0; kk < K; ++kk) vpf[i * K + kk] = a.V[kk * pb.nv + pb.ncp + i];
    for (int i = threadIdx.x; i <= pb.ncorr; i += blockDim.x) coff[i] = (int)pb.corr_off[i];
    if (lane == 0) {
        mbar_init(&bars[2 * wid], 1);
        mbar_init(&bars[2 * wid + 1], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();

    const uint32_t occ_b = (uint32_t)a.Nst, cid_b = (uint32_t)a.ncst * 2u;
    const uint32_t pf_b = (uint32_t)(a.Pst * a.st_bytes);
    unsigned char* const mybuf0 = bufs + (size_t)(2 * wid) * a.buf_bytes;
    const int64_t stride = (int64_t)gridDim.x * nw;
    const int64_t s0 = (int64_t)blockIdx.x * nw + wid;

    auto issue = [&](int64_t s, int b) {
        unsigned char* d = mybuf0 + (size_t)b * a.buf_bytes;
        mbar_expect_tx(&bars[2 * wid + b], occ_b + cid_b + pf_b);
        bulk_g2s(d, a.s_occ + s * a.Nst, occ_b, &bars[2 * wid + b]);
        bulk_g2s(d + occ_b, a.s_cidx + s * a.ncst, cid_b, &bars[2 * wid + b]);
        bulk_g2s(d + occ_b + cid_b, (const unsigned char*)a.s_pf + s * (int64_t)pf_b, pf_b, &bars[2 * wid + b]);
    };
    if (lane == 0) {
        if (s0 < a.n_s) issue(s0, 0);
        if (s0 + stride < a.n_s) issue(s0 + stride, 1);
    }
    __syncwarp();

    const int P_uu = nu * (nu - 1) / 2, P_dd = nd * (nd - 1) / 2;
    bool timed_out = false;
    int it = 0;
    for (int64_t s = s0; s < a.n_s; s += stride, ++it) {
        const int b = it & 1;
        const uint32_t par = (uint32_t)((it >> 1) & 1);
        if (!mbar_wait_bounded(&bars[2 * wid + b], par)) { timed_out = true; break; }
        const unsigned char* buf = mybuf0 + (size_t)b * a.buf_bytes;
        const uint8_t* occ = buf;
        const uint16_t* cid = (const uint16_t*)(buf + occ_b);
        const ST* W = (const ST*)(buf + occ_b + cid_b);
        const int ou = lane < nu ? (int)occ[lane] : 0;
        const int od = lane < nd ? (int)occ[nu + lane] : 0;
        float t[K];
#pragma unroll
        for (int kk = 0; kk < K; ++kk) t[kk] = 0.f;
        for (int c = lane; c < pb.ncorr; c += 32) {
            const int k = coff[c] + cid[c];
            const float ic = __ldg(a.invC + k);
#pragma unroll
            for (int kk = 0; kk < K; ++kk) t[kk] += __ldg(a.V + kk * pb.nv + k) * ic;
        }
        tri_block<ST, K, 0>(W, 0, nu, ou, M, vpf, acc, t);
        tri_block<ST, K, 0>(W, P_uu, nd, od, M, vpf, acc, t);
        rect_block<ST, K, 0>(W, P_uu + P_dd, nu, nd, ou, od, M, vpf, acc, t);
#pragma unroll
        for (int kk = 0; kk < K; ++kk) t[kk] = warp_sum(t[kk]);
        if (lane == 0)
#pragma unroll
            for (int kk = 0; kk < K; ++kk) a.T[s * K + kk] = t[kk];
        tri_block<ST, K, 1>(W, 0, nu, ou, M, vpf, acc, t);
        tri_block<ST, K, 1>(W, P_uu, nd, od, M, vpf, acc, t);
        rect_block<ST, K, 1>(W, P_uu + P_dd, nu, nd, ou, od, M, vpf, acc, t);
        __syncwarp();
        if (lane == 0 && s + 2 * stride < a.n_s) {
            // order this warp's generic reads of the buffer before the async refill
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(s + 2 * stride, b);
        }
        __syncwarp();
    }
    if (timed_out) {
        if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
        // drain the copies still addressed to this warp's buffers (bounded)
        for (int j = 0; j < 2; ++j) {
            const int u = it + j;
            mbar_wait_bounded(&bars[2 * wid + (u & 1)], (uint32_t)((u >> 1) & 1));
        }
    }
    __syncthreads();
    float* dst = a.pf_partial + (size_t)blockIdx.x * npf * K;
    for (int i = threadIdx.x; i < npf * K; i += blockDim.x) dst[i] = acc[i];
}

template __global__ void k_sr_stream<__nv_bfloat16, 1>(StreamArgs);
template __global__ void k_sr_stream<__nv_bfloat16, 2>(StreamArgs);
template __global__ void k_sr_stream<float, 1>(StreamArgs);
template __global__ void k_sr_stream<float, 2>(StreamArgs);

}  // namespace vmc
