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
#include "tma.cuh"

namespace vmc {

template <typename ST> __device__ __forceinline__ float ld_w(const ST* w, int i);
template <> __device__ __forceinline__ float ld_w<float>(const float* w, int i) { return w[i]; }
template <> __device__ __forceinline__ float ld_w<__nv_bfloat16>(const __nv_bfloat16* w, int i) {
    return __bfloat162float(w[i]);
}

__device__ __forceinline__ int rowbase_of(int p, int M) { return ((p * (2 * M - 3 - p)) >> 1) - 1; }

// Lane tables for the two triangles, built once per CTA: entry (it, lane) of
// a triangle with n electrons is the pair (r, b) that lane handles in folded
// iteration it (row it together with row n-2-it) and its offset inside the
// triangle, packed as e | r << 16 | b << 24, or ~0u when the lane idles.
__device__ __forceinline__ uint32_t tri_entry(int n, int it, int lane) {
    const int r1 = it, r2 = n - 2 - it;
    int r, b;
    bool valid = lane < n;
    if (lane > r1) { r = r1; b = lane; }
    else { r = r2; b = r2 + 1 + lane; valid = valid && (r1 < r2); }
    if (b >= n) valid = false;
    if (!valid) return ~0u;
    const int e = r * n - ((r * (r + 1)) >> 1) + (b - r - 1);
    return (uint32_t)e | ((uint32_t)r << 16) | ((uint32_t)b << 24);
}

// One triangle (spin block with n electrons whose ascending orbitals sit in
// register `o` of lanes 0..n-1 and their row bases f_pq index - q in `rbo`,
// block offset off).  PHASE 0 gathers into t (branch-free: idle lanes read
// element 0 / parameter 0 with weight 0, two partial sums per vector), PHASE 1
// scatters t into acc with predicated shared atomics.
template <typename ST, int K, int PHASE>
__device__ __forceinline__ void tri_row(const ST* W, int off, const uint32_t* tab, int i, int o, int rbo,
                                        const float* vpf, float* acc, const float (&t)[K], float (&ta)[K]) {
    const int lane = threadIdx.x & 31;
    const uint32_t en = tab[i * 32 + lane];
    const bool valid = en != ~0u;
    const uint32_t enz = valid ? en : 0u;
    const int rb = __shfl_sync(VMC_FULL_MASK, rbo, (int)((enz >> 16) & 255u));
    const int q = __shfl_sync(VMC_FULL_MASK, o, (int)(enz >> 24));
    const int pq = valid ? rb + q : 0;
    const float w = valid ? ld_w<ST>(W, off + (int)(enz & 0xFFFFu)) : 0.f;
    if (PHASE == 0) {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) ta[kk] += w * vpf[pq * K + kk];
    } else if (valid) {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) atomicAdd(&acc[pq * K + kk], t[kk] * w);
    }
}

// One triangle (spin block with n electrons whose ascending orbitals sit in
// register `o` of lanes 0..n-1 and their f_pq row bases in `rbo`, block
// offset off), two folded rows per step into two partial sums.  PHASE 0
// gathers into t (branch-free: idle lanes read element 0 / parameter 0 with
// weight 0), PHASE 1 scatters t into acc with predicated shared atomics.
template <typename ST, int K, int PHASE>
__device__ __forceinline__ void tri_block(const ST* W, int off, int n, const uint32_t* tab, int o, int rbo,
                                          const float* vpf, float* acc, float (&t)[K]) {
    const int iters = n >> 1;
    float t0[K], t1[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) t0[kk] = t1[kk] = 0.f;
    int i = 0;
    for (; i + 1 < iters; i += 2) {
        tri_row<ST, K, PHASE>(W, off, tab, i, o, rbo, vpf, acc, t, t0);
        tri_row<ST, K, PHASE>(W, off, tab, i + 1, o, rbo, vpf, acc, t, t1);
    }
    if (i < iters) tri_row<ST, K, PHASE>(W, off, tab, i, o, rbo, vpf, acc, t, t0);
    if (PHASE == 0)
#pragma unroll
        for (int kk = 0; kk < K; ++kk) t[kk] += t0[kk] + t1[kk];
}

template <typename ST, int K, int PHASE>
__device__ __forceinline__ void rect_row(const ST* Wl, int r, int stride, bool lane_ok, int rbu, int od,
                                         const float* vpf, float* acc, const float (&t)[K], float (&ta)[K]) {
    const int rb = __shfl_sync(VMC_FULL_MASK, rbu, r);
    const int pq = lane_ok ? rb + od : 0;
    const float w = lane_ok ? ld_w<ST>(Wl, r * stride) : 0.f;
    if (PHASE == 0) {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) ta[kk] += w * vpf[pq * K + kk];
    } else if (lane_ok) {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) atomicAdd(&acc[pq * K + kk], t[kk] * w);
    }
}

template <typename ST, int K, int PHASE>
__device__ __forceinline__ void rect_block(const ST* W, int off, int nu, int nd, int rbu, int od,
                                           const float* vpf, float* acc, float (&t)[K]) {
    const int lane = threadIdx.x & 31;
    const bool lane_ok = lane < nd;
    const ST* Wl = W + off + (lane_ok ? lane : 0);
    const int stride = lane_ok ? nd : 0;
    float t0[K], t1[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) t0[kk] = t1[kk] = 0.f;
    int r = 0;
    for (; r + 1 < nu; r += 2) {
        rect_row<ST, K, PHASE>(Wl, r, stride, lane_ok, rbu, od, vpf, acc, t, t0);
        rect_row<ST, K, PHASE>(Wl, r + 1, stride, lane_ok, rbu, od, vpf, acc, t, t1);
    }
    if (r < nu) rect_row<ST, K, PHASE>(Wl, r, stride, lane_ok, rbu, od, vpf, acc, t, t0);
    if (PHASE == 0)
#pragma unroll
        for (int kk = 0; kk < K; ++kk) t[kk] += t0[kk] + t1[kk];
}

template <typename ST, int K>
__global__ void __launch_bounds__(768, 1) k_sr_stream(StreamArgs a) {
    if (a.stop && *a.stop) return;
    extern __shared__ __align__(128) unsigned char smem[];
    const DevProblem& pb = a.pb;
    const int npf = pb.npf, M = pb.M, nu = pb.nu, nd = pb.nd;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // layout: acc | vpf | corr offsets | lane tables | mbarriers | staging buffers
    float* acc = (float*)smem;
    float* vpf = acc + (size_t)npf * K;
    int* coff = (int*)(vpf + (size_t)npf * K);
    uint32_t* tab_u = (uint32_t*)(coff + pb.ncorr + 1);
    uint32_t* tab_d = tab_u + (nu >> 1) * 32;
    uint64_t* bars = (uint64_t*)(((uintptr_t)(tab_d + (nd >> 1) * 32) + 15) & ~(uintptr_t)15);
    unsigned char* bufs = (unsigned char*)(((uintptr_t)(bars + 2 * nw) + 127) & ~(uintptr_t)127);

    for (int i = threadIdx.x; i < npf * K; i += blockDim.x) acc[i] = 0.f;
    for (int i = threadIdx.x; i < npf; i += blockDim.x)
#pragma unroll
        for (int kk = 0; kk < K; ++kk) vpf[i * K + kk] = a.V[kk * pb.nv + pb.ncp + i];
    for (int i = threadIdx.x; i <= pb.ncorr; i += blockDim.x) coff[i] = (int)pb.corr_off[i];
    for (int i = threadIdx.x; i < (nu >> 1) * 32; i += blockDim.x) tab_u[i] = tri_entry(nu, i >> 5, i & 31);
    for (int i = threadIdx.x; i < (nd >> 1) * 32; i += blockDim.x) tab_d[i] = tri_entry(nd, i >> 5, i & 31);
    if (lane == 0) {
        mbar_init(&bars[2 * wid], 1);
        mbar_init(&bars[2 * wid + 1], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();

    const uint32_t occ_b = (uint32_t)a.Nst;
    const uint32_t pf_b = (uint32_t)(a.Pst * a.st_bytes);
    unsigned char* const mybuf0 = bufs + (size_t)(2 * wid) * a.buf_bytes;
    const int64_t stride = (int64_t)gridDim.x * nw;
    const int64_t s0 = (int64_t)blockIdx.x * nw + wid;

    auto issue = [&](int64_t s, int b) {
        unsigned char* d = mybuf0 + (size_t)b * a.buf_bytes;
        mbar_expect_tx(&bars[2 * wid + b], occ_b + pf_b);
        bulk_g2s(d, a.s_occ + s * a.Nst, occ_b, &bars[2 * wid + b]);
        bulk_g2s(d + occ_b, (const unsigned char*)a.s_pf + s * (int64_t)pf_b, pf_b, &bars[2 * wid + b]);
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
        // correlator part of the gather straight from global memory while the
        // record is in flight
        float t[K];
#pragma unroll
        for (int kk = 0; kk < K; ++kk) t[kk] = 0.f;
        const cstate_t* cid = a.s_cidx + s * a.ncst;
        for (int c = lane; c < pb.ncorr; c += 32) {
            const int k = coff[c] + (int)__ldg(cid + c);
            const float ic = __ldg(a.invC + k);
#pragma unroll
            for (int kk = 0; kk < K; ++kk) t[kk] += __ldg(a.V + kk * pb.nv + k) * ic;
        }
        if (!mbar_wait_limit(&bars[2 * wid + b], (uint32_t)((it >> 1) & 1), a.spin_limit)) { timed_out = true; break; }
        const unsigned char* buf = mybuf0 + (size_t)b * a.buf_bytes;
        const uint8_t* occ = buf;
        const ST* W = (const ST*)(buf + occ_b);
        const int ou = lane < nu ? (int)occ[lane] : 0;
        const int od = lane < nd ? (int)occ[nu + lane] : 0;
        const int rbu = rowbase_of(ou, M), rbd = rowbase_of(od, M);
        tri_block<ST, K, 0>(W, 0, nu, tab_u, ou, rbu, vpf, acc, t);
        tri_block<ST, K, 0>(W, P_uu, nd, tab_d, od, rbd, vpf, acc, t);
        rect_block<ST, K, 0>(W, P_uu + P_dd, nu, nd, rbu, od, vpf, acc, t);
#pragma unroll
        for (int kk = 0; kk < K; ++kk) t[kk] = warp_sum(t[kk]);
        if (lane == 0)
#pragma unroll
            for (int kk = 0; kk < K; ++kk) a.T[s * K + kk] = t[kk];
        tri_block<ST, K, 1>(W, 0, nu, tab_u, ou, rbu, vpf, acc, t);
        tri_block<ST, K, 1>(W, P_uu, nd, tab_d, od, rbd, vpf, acc, t);
        rect_block<ST, K, 1>(W, P_uu + P_dd, nu, nd, rbu, od, vpf, acc, t);
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

// BF16 store, one vector: every element the gather touches is cached in one
// register, (pq << 16) | bf16 bits, so the scatter is unpack + multiply +
// shared atomic.  Slots 0..15 hold the folded up-up rows, 16..31 the folded
// down-down rows, 32..63 the up-down rows (electrons per spin <= 32).
__global__ void __launch_bounds__(512, 1) k_sr_stream_bf16c(StreamArgs a) {
    if (a.stop && *a.stop) return;
    extern __shared__ __align__(128) unsigned char smem[];
    const DevProblem& pb = a.pb;
    const int npf = pb.npf, M = pb.M, nu = pb.nu, nd = pb.nd;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float* acc = (float*)smem;
    float* vpf = acc + npf;
    int* coff = (int*)(vpf + npf);
    uint32_t* tab_u = (uint32_t*)(coff + pb.ncorr + 1);
    uint32_t* tab_d = tab_u + (nu >> 1) * 32;
    uint64_t* bars = (uint64_t*)(((uintptr_t)(tab_d + (nd >> 1) * 32) + 15) & ~(uintptr_t)15);
    unsigned char* bufs = (unsigned char*)(((uintptr_t)(bars + 2 * nw) + 127) & ~(uintptr_t)127);

    for (int i = threadIdx.x; i < npf; i += blockDim.x) {
        acc[i] = 0.f;
        vpf[i] = a.V[pb.ncp + i];
    }
    for (int i = threadIdx.x; i <= pb.ncorr; i += blockDim.x) coff[i] = (int)pb.corr_off[i];
    for (int i = threadIdx.x; i < (nu >> 1) * 32; i += blockDim.x) tab_u[i] = tri_entry(nu, i >> 5, i & 31);
    for (int i = threadIdx.x; i < (nd >> 1) * 32; i += blockDim.x) tab_d[i] = tri_entry(nd, i >> 5, i & 31);
    if (lane == 0) {
        mbar_init(&bars[2 * wid], 1);
        mbar_init(&bars[2 * wid + 1], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncthreads();

    const uint32_t occ_b = (uint32_t)a.Nst;
    const uint32_t pf_b = (uint32_t)(a.Pst * 2);
    unsigned char* const mybuf0 = bufs + (size_t)(2 * wid) * a.buf_bytes;
    const int64_t stride = (int64_t)gridDim.x * nw;
    const int64_t s0 = (int64_t)blockIdx.x * nw + wid;
    auto issue = [&](int64_t s, int b) {
        unsigned char* d = mybuf0 + (size_t)b * a.buf_bytes;
        mbar_expect_tx(&bars[2 * wid + b], occ_b + pf_b);
        bulk_g2s(d, a.s_occ + s * a.Nst, occ_b, &bars[2 * wid + b]);
        bulk_g2s(d + occ_b, (const unsigned char*)a.s_pf + s * (int64_t)pf_b, pf_b, &bars[2 * wid + b]);
    };
    if (lane == 0) {
        if (s0 < a.n_s) issue(s0, 0);
        if (s0 + stride < a.n_s) issue(s0 + stride, 1);
    }
    __syncwarp();

    const int P_uu = nu * (nu - 1) / 2, P_dd = nd * (nd - 1) / 2;
    const int iu = nu >> 1, id = nd >> 1;
    bool timed_out = false;
    int it = 0;
    for (int64_t s = s0; s < a.n_s; s += stride, ++it) {
        const int b = it & 1;
        float t = 0.f;
        const cstate_t* cid = a.s_cidx + s * a.ncst;
        for (int c = lane; c < pb.ncorr; c += 32) {
            const int k = coff[c] + (int)__ldg(cid + c);
            t += __ldg(a.V + k) * __ldg(a.invC + k);
        }
        if (!mbar_wait_limit(&bars[2 * wid + b], (uint32_t)((it >> 1) & 1), a.spin_limit)) { timed_out = true; break; }
        const unsigned char* buf = mybuf0 + (size_t)b * a.buf_bytes;
        const uint16_t* W = (const uint16_t*)(buf + occ_b);
        const int ou = lane < nu ? (int)buf[lane] : 0;
        const int od = lane < nd ? (int)buf[nu + lane] : 0;
        const int rbu = rowbase_of(ou, M), rbd = rowbase_of(od, M);
        // branch-free gather: idle lanes read element 0 / parameter 0 with a
        // zero weight; four partial sums keep the FMA chains independent
        uint32_t cache[64];
        float ta[4] = {t, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            cache[i] = ~0u;
            if (i < iu) {
                const uint32_t en = tab_u[i * 32 + lane];
                const bool valid = en != ~0u;
                const uint32_t enz = valid ? en : 0u;
                const int rb = __shfl_sync(VMC_FULL_MASK, rbu, (int)((enz >> 16) & 255u));
                const int q = __shfl_sync(VMC_FULL_MASK, ou, (int)(enz >> 24));
                const int pq = valid ? rb + q : 0;
                const uint32_t wr = valid ? (uint32_t)W[enz & 0xFFFFu] : 0u;
                ta[i & 3] += __uint_as_float(wr << 16) * vpf[pq];
                cache[i] = valid ? (((uint32_t)pq << 16) | wr) : ~0u;
            }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            cache[16 + i] = ~0u;
            if (i < id) {
                const uint32_t en = tab_d[i * 32 + lane];
                const bool valid = en != ~0u;
                const uint32_t enz = valid ? en : 0u;
                const int rb = __shfl_sync(VMC_FULL_MASK, rbd, (int)((enz >> 16) & 255u));
                const int q = __shfl_sync(VMC_FULL_MASK, od, (int)(enz >> 24));
                const int pq = valid ? rb + q : 0;
                const uint32_t wr = valid ? (uint32_t)W[P_uu + (enz & 0xFFFFu)] : 0u;
                ta[i & 3] += __uint_as_float(wr << 16) * vpf[pq];
                cache[16 + i] = valid ? (((uint32_t)pq << 16) | wr) : ~0u;
            }
        }
        const bool lane_ud = lane < nd;
        const uint16_t* Wud = W + P_uu + P_dd + (lane_ud ? lane : 0);
        const int stride_ud = lane_ud ? nd : 0;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            cache[32 + r] = ~0u;
            if (r < nu) {
                const int rb = __shfl_sync(VMC_FULL_MASK, rbu, r);
                const int pq = lane_ud ? rb + od : 0;
                const uint32_t wr = lane_ud ? (uint32_t)Wud[r * stride_ud] : 0u;
                ta[r & 3] += __uint_as_float(wr << 16) * vpf[pq];
                cache[32 + r] = lane_ud ? (((uint32_t)pq << 16) | wr) : ~0u;
            }
        }
        t = (ta[0] + ta[1]) + (ta[2] + ta[3]);
        t = warp_sum(t);
        if (lane == 0) a.T[s] = t;
#pragma unroll
        for (int i = 0; i < 64; ++i) {
            const uint32_t c = cache[i];
            if (c != ~0u) atomicAdd(&acc[c >> 16], t * __uint_as_float(c << 16));
        }
        __syncwarp();
        if (lane == 0 && s + 2 * stride < a.n_s) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(s + 2 * stride, b);
        }
        __syncwarp();
    }
    if (timed_out) {
        if (lane == 0) atomicOr(a.status, ST_TIMEOUT);
        for (int j = 0; j < 2; ++j) {
            const int u = it + j;
            mbar_wait_bounded(&bars[2 * wid + (u & 1)], (uint32_t)((u >> 1) & 1));
        }
    }
    __syncthreads();
    float* dst = a.pf_partial + (size_t)blockIdx.x * npf;
    for (int i = threadIdx.x; i < npf; i += blockDim.x) dst[i] = acc[i];
}

template __global__ void k_sr_stream<__nv_bfloat16, 1>(StreamArgs);
template __global__ void k_sr_stream<__nv_bfloat16, 2>(StreamArgs);
template __global__ void k_sr_stream<float, 1>(StreamArgs);
template __global__ void k_sr_stream<float, 2>(StreamArgs);

}  // namespace vmc
