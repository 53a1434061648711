// Sorted two-pass Eq. 7 product for the BF16 store.
//
// The per-sample pass with shared-memory scatter is bound by shared atomics
// and index arithmetic (every pairing element of every sample costs an
// occupation lookup and a shared atomic).  Because the O store is fixed for
// all CG iterations of an SR step, the index work is done once per step:
//
//   G  [n_s][Pst] u32   (pq << 16) | bf16 value, sample-major: the gather
//      t_s = sum_e W_e v[pq(e)] is a pure stream with a shared-memory lookup of
//      v and no atomics;
//   T  u32 entries (s_local << 16) | bf16 value, parameter-major per chunk of
//      at most 65,536 samples (a counting sort of G by pq), each run padded to
//      whole 128-entry blocks and interleaved inside a block: the scatter
//      out[pq] = sum_s t_s W_s[pq] is one warp per parameter summing a
//      contiguous run, with no atomics and no per-CTA partial images.
//
// The build (count, scan, fill) streams G three times once per SR step.
#include "common.cuh"
#include "kernels.h"
#include "corr_runs.cuh"

namespace vmc {

// G rows: the P pairing elements of a sample as (pq << 16) | bf16, cut into
// kGParts parts of consecutive pq (part f holds the elements of full-matrix
// row-major rank f QE .. (f+1) QE - 1 over ascending positions, which is pq
// order, QE = ceil(P / kGParts)), each part in a region of WQ = ceil(QE / 4)
// 16-byte words, so the row stride is kGParts * WQ * 4 entries.  The
// single-pass product gives each part to one warp of a group, and the parts'
// pq ranges are disjoint.
//
// Inside a part the elements are placed in a bank-aware order.  A reader's
// lane L holds word L + 32 u of the region and looks up v[pq] in shared
// memory for element j of it, so the 32 lanes of one lookup instruction
// (u, j) read the region slots 128 u + 4 L + j.  Lookups whose pq fall in the
// same shared-memory bank (pq mod 32) at different addresses serialise, and
// random pq give about 3.5-way conflicts.  So the elements of a part are
// ranked within their bank and placed in rank-major order (rank 0 of every
// bank, then rank 1, ...) along the instruction groups: a group holds at
// most two elements of a bank.  Padding slots hold (0, 0.0); parts whose
// largest bank count exceeds kBankRanks keep the plain order.
constexpr int kBankRanks = 128;

// region position of slot k in the reader's instruction-group order
__device__ __forceinline__ int group_slot_pos(int k, int n4) {
    const int nfull = n4 >> 5, m = n4 & 31;
    if (k < 128 * nfull) return 128 * (k >> 7) + 4 * (k & 31) + ((k >> 5) & 3);
    const int kr = k - 128 * nfull;
    return 128 * nfull + 4 * (kr % m) + kr / m;
}

// fulltab[r] = e | a << 16 | b << 24: rank r in the full row-major order over
// positions a < b, and e the element's index in the store's block order
__global__ void __launch_bounds__(256) k_build_G(DevProblem pb, int64_t n_s, const uint8_t* s_occ, int Nst,
                                                 const __nv_bfloat16* pf16, int64_t Pst, const uint32_t* fulltab,
                                                 int wq, int64_t Gst, uint32_t* G) {
    __shared__ uint8_t occw[8][64];
    __shared__ uint32_t cnt[8][32];
    __shared__ uint32_t msk[8][kBankRanks];
    __shared__ uint16_t rbase[8][kBankRanks];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t s = (int64_t)blockIdx.x * 8 + wid;
    if (s >= n_s) return;
    for (int i = lane; i < pb.N; i += 32) occw[wid][i] = s_occ[s * Nst + i];
    __syncwarp();
    const uint16_t* src = (const uint16_t*)(pf16 + s * Pst);
    const int P = pb.P, QE = (P + kGParts - 1) / kGParts;
    for (int f = 0; f < kGParts; ++f) {
        uint32_t* dst = G + s * Gst + (int64_t)f * wq * 4;
        const int r0 = f * QE, r1 = min(P, r0 + QE), n = max(0, r1 - r0);
        cnt[wid][lane] = 0u;
        __syncwarp();
        for (int r = r0 + lane; r < r1; r += 32) {
            const uint32_t ft = fulltab[r];
            const int pq = (int)pf_row_base(pb.M, occw[wid][(ft >> 16) & 255]) + occw[wid][ft >> 24];
            atomicAdd(&cnt[wid][pq & 31], 1u);
        }
        __syncwarp();
        const uint32_t c = cnt[wid][lane];
        uint32_t maxc = c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) maxc = max(maxc, __shfl_xor_sync(0xffffffffu, maxc, o));
        const bool ranked = maxc <= (uint32_t)kBankRanks;
        if (ranked) {
            // banks with more than r elements, and the slots before rank r
            for (int r = 0; r < (int)maxc; ++r) {
                const uint32_t m = __ballot_sync(0xffffffffu, c > (uint32_t)r);
                if (lane == 0) msk[wid][r] = m;
            }
            __syncwarp();
            if (lane == 0) {
                uint32_t run = 0;
                for (int r = 0; r < (int)maxc; ++r) {
                    rbase[wid][r] = (uint16_t)run;
                    run += __popc(msk[wid][r]);
                }
            }
            cnt[wid][lane] = 0u;
            __syncwarp();
        }
        for (int r = r0 + lane; r < r1; r += 32) {
            const uint32_t ft = fulltab[r];
            const int pq = (int)pf_row_base(pb.M, occw[wid][(ft >> 16) & 255]) + occw[wid][ft >> 24];
            const uint32_t g = ((uint32_t)pq << 16) | (uint32_t)src[ft & 0xFFFFu];
            int slot = r - r0;
            if (ranked) {
                const int b = pq & 31;
                const uint32_t k = atomicAdd(&cnt[wid][b], 1u);
                slot = rbase[wid][k] + __popc(msk[wid][k] & ((1u << b) - 1u));
            }
            dst[group_slot_pos(slot, wq)] = g;
        }
        for (int k = n + lane; k < 4 * wq; k += 32) dst[group_slot_pos(k, wq)] = 0u;
        __syncwarp();
    }
}

// Block b of a chunk [s_begin, s_end) owns samples s_begin + [b*per, (b+1)*per).
__device__ __forceinline__ void block_range(int64_t s_begin, int64_t s_end, int nblk, int64_t* lo, int64_t* hi) {
    const int64_t n = s_end - s_begin;
    const int64_t per = (n + nblk - 1) / nblk;
    *lo = s_begin + min(n, (int64_t)blockIdx.x * per);
    *hi = s_begin + min(n, (int64_t)(blockIdx.x + 1) * per);
}

// counts[b][pq] = occurrences of pq in block b's samples
__global__ void __launch_bounds__(512) k_count_G(const uint32_t* G, int64_t Pst, int P, int64_t s_begin,
                                                 int64_t s_end, int npf, uint32_t* counts) {
    extern __shared__ uint32_t cnt[];
    for (int i = threadIdx.x; i < npf; i += blockDim.x) cnt[i] = 0u;
    __syncthreads();
    int64_t lo, hi;
    block_range(s_begin, s_end, gridDim.x, &lo, &hi);
    for (int64_t s = lo; s < hi; ++s) {
        const uint32_t* g = G + s * Pst;
        for (int e = threadIdx.x; e < Pst; e += blockDim.x) {
            const uint32_t v = g[e];
            if (v) atomicAdd(&cnt[v >> 16], 1u);   // padding (and exact zeros) carry nothing
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npf; i += blockDim.x) counts[(size_t)blockIdx.x * npf + i] = cnt[i];
}

// per parameter: running offsets over the blocks (in place) and the run
// length padded to a whole number of kTRun-entry blocks
__global__ void k_scan_blocks(uint32_t* counts, int nblk, int npf, uint32_t* total) {
    const int pq = blockIdx.x * blockDim.x + threadIdx.x;
    if (pq >= npf) return;
    uint32_t run = 0u;
    for (int b = 0; b < nblk; ++b) {
        const uint32_t c = counts[(size_t)b * npf + pq];
        counts[(size_t)b * npf + pq] = run;
        run += c;
    }
    total[pq] = (run + kTRun - 1) / kTRun * kTRun;
}

// Position inside a run of logical entry r.  Within each kTRun = 128 entry
// block, entry 32 j + L sits at 4 L + j, so lane L's 16-byte word holds
// entries L, L + 32, L + 64, L + 96 and the j-th lookup instruction of the
// scatter covers 32 consecutive entries (consecutive, sorted samples: a few
// cache lines instead of 32).
__device__ __forceinline__ uint32_t run_slot(uint32_t r) {
    return (r & ~(uint32_t)(kTRun - 1)) + 4u * (r & 31u) + ((r >> 5) & 3u);
}

// base[pq] = exclusive prefix of total over pq (single block), base[npf] = sum
__global__ void __launch_bounds__(1024) k_scan_params(const uint32_t* total, int npf, uint32_t base0,
                                                      uint32_t* base) {
    __shared__ uint32_t part[1024];
    const int per = (npf + blockDim.x - 1) / blockDim.x;
    const int lo = threadIdx.x * per, hi = min(npf, lo + per);
    uint32_t s = 0u;
    for (int i = lo; i < hi; ++i) s += total[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        uint32_t v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = base0 + (threadIdx.x ? part[threadIdx.x - 1] : 0u);
    for (int i = lo; i < hi; ++i) {
        base[i] = run;
        run += total[i];
    }
    if (threadIdx.x == blockDim.x - 1) base[npf] = base0 + part[blockDim.x - 1];
}

// T[base[pq] + run_slot(offset[b][pq] + k)] = (s - s_begin) << 16 | bf16, in
// block order; the padding of each run stays zero (weight 0)
__global__ void __launch_bounds__(512) k_fill_T(const uint32_t* G, int64_t Pst, int P, int64_t s_begin,
                                                int64_t s_end, int npf, const uint32_t* offs, const uint32_t* base,
                                                uint32_t* T) {
    extern __shared__ uint32_t cur[];
    uint32_t* rb = cur + npf;
    for (int i = threadIdx.x; i < npf; i += blockDim.x) {
        cur[i] = offs[(size_t)blockIdx.x * npf + i];
        rb[i] = base[i];
    }
    __syncthreads();
    int64_t lo, hi;
    block_range(s_begin, s_end, gridDim.x, &lo, &hi);
    for (int64_t s = lo; s < hi; ++s) {
        const uint32_t* g = G + s * Pst;
        const uint32_t sl = (uint32_t)(s - s_begin) << 16;
        for (int e = threadIdx.x; e < Pst; e += blockDim.x) {
            const uint32_t v = g[e];
            if (!v) continue;
            const uint32_t pq = v >> 16;
            const uint32_t r = atomicAdd(&cur[pq], 1u);
            T[rb[pq] + run_slot(r)] = sl | (v & 0xFFFFu);
        }
    }
}

// Correlator runs: the samples of each correlator parameter, grouped by
// parameter (class block off_q + state), built once per set of samples from
// the transposed state array.  Grid (class, slice): a CTA counts the states
// of its class's correlators over one slice of the samples in shared memory
// and adds its counts to the global ones (a class shared by many correlators
// spreads over many CTAs); the fill then places every entry through global
// cursors.  A sample appears once per correlator of the class in that state.
__device__ __forceinline__ void corr_slice(int64_t n_s, int nsl, int64_t* s0, int64_t* s1) {
    const int64_t per = (n_s + nsl - 1) / nsl;
    *s0 = min(n_s, (int64_t)blockIdx.y * per);
    *s1 = min(n_s, *s0 + per);
}

// shared_hist = 0 (classes of more states than shared memory holds): count
// straight into the global counters
__global__ void __launch_bounds__(512) k_count_C(DevProblem pb, int64_t n_s, const cstate_t* cidxT,
                                                 uint32_t* ccount, int shared_hist) {
    extern __shared__ uint32_t hist[];
    const int q = blockIdx.x;
    const int64_t off = pb.class_off[q];
    const int d = (int)(pb.class_off[q + 1] - off);
    if (shared_hist) {
        for (int i = threadIdx.x; i < d; i += blockDim.x) hist[i] = 0u;
        __syncthreads();
    }
    int64_t s0, s1;
    corr_slice(n_s, gridDim.y, &s0, &s1);
    for (int j = pb.class_ptr[q]; j < pb.class_ptr[q + 1]; ++j) {
        const cstate_t* st = cidxT + (int64_t)pb.class_inst[j] * n_s;
        for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
            if (shared_hist) atomicAdd(&hist[st[s]], 1u);
            else atomicAdd(&ccount[off + st[s]], 1u);
        }
    }
    if (shared_hist) {
        __syncthreads();
        for (int i = threadIdx.x; i < d; i += blockDim.x)
            if (hist[i]) atomicAdd(&ccount[off + i], hist[i]);
    }
}

// cursor[k] starts at the run start of parameter k (a copy of cbase)
__global__ void __launch_bounds__(512) k_fill_C(DevProblem pb, int64_t n_s, const cstate_t* cidxT,
                                                uint32_t* cursor, uint32_t* Tc) {
    const int q = blockIdx.x;
    const int64_t off = pb.class_off[q];
    int64_t s0, s1;
    corr_slice(n_s, gridDim.y, &s0, &s1);
    // entry = sample << 5 | (parameter index mod 32): the scatter's warps own
    // 32 consecutive parameters and sum each one's contiguous segment
    for (int j = pb.class_ptr[q]; j < pb.class_ptr[q + 1]; ++j) {
        const cstate_t* st = cidxT + (int64_t)pb.class_inst[j] * n_s;
        for (int64_t s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
            const uint32_t state = st[s];
            Tc[atomicAdd(&cursor[off + state], 1u)] = ((uint32_t)s << 5) | (uint32_t)((off + state) & 31);
        }
    }
}

// Work items of the correlator scatter: group g (parameters 32 g .. 32 g + 31,
// one contiguous stretch of entries) is cut into pieces of at most
// kCorrItem entries.  n_items[g] then its exclusive scan give item_base.
__global__ void k_corr_item_count(const uint32_t* cbase, int64_t ncp, uint32_t* n_items) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ng = (ncp + 31) / 32;
    if (g >= ng) return;
    const uint32_t len = cbase[min(ncp, 32 * g + 32)] - cbase[32 * g];
    n_items[g] = len == 0 ? 1u : (len + kCorrItem - 1) / kCorrItem;
}

__global__ void k_corr_item_fill(const uint32_t* cbase, int64_t ncp, const uint32_t* item_base, uint2* items) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ng = (ncp + 31) / 32;
    if (g >= ng) return;
    const uint32_t e0 = cbase[32 * g], e1 = cbase[min(ncp, 32 * g + 32)];
    uint32_t i = item_base[g];
    for (uint32_t e = e0; e == e0 || e < e1; e += kCorrItem) items[i++] = make_uint2((uint32_t)g, e);
}

// gather: t_s = sum_c V[k_c]/C[k_c] + sum_e W_e v[pq(e)] - Obar . V, warp per
// sample.  Centering t_s makes the scatter produce the covariance
// (1/n) sum_s (t_s - Obar . V) O_s = S V directly, with no cancellation
// between <O (O . V)> and Obar (Obar . V).  U = ceil(Pst / 128): every lane
// holds its U 16-byte words of a row, and the warp loads its next row while
// it works on the current one, so a whole row (6 KB at 56 electrons) is
// always in flight per warp.
template <int K, int U>
__global__ void __launch_bounds__(gather_threads(K)) k_gather_G(SortedArgs a) {
    if (a.stop && *a.stop) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const DevProblem& pb = a.pb;
    float* vpf = (float*)smem;
    int* coff = (int*)(vpf + (size_t)pb.npf * K);
    for (int i = threadIdx.x; i < pb.npf; i += blockDim.x)
#pragma unroll
        for (int kk = 0; kk < K; ++kk) vpf[i * K + kk] = a.V[kk * pb.nv + pb.ncp + i];
    for (int i = threadIdx.x; i <= pb.ncorr; i += blockDim.x) coff[i] = (int)pb.corr_off[i];
    __shared__ float obv[K];
    if (threadIdx.x < 32) {
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const double c = warp_sum_partials(a.obv_part, a.n_obv_part, kk, K);
            if (threadIdx.x == 0) obv[kk] = (float)c;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int n4 = (int)(a.Pst >> 2);
    double tt = 0.0;   // lane 0: sum of the warp's centered t_s^2
    const int64_t gstride = (int64_t)gridDim.x * nw;
    uint4 g[U];
    {
        const int64_t s = (int64_t)blockIdx.x * nw + wid;
        const uint4* g4 = (const uint4*)(a.G + s * a.Pst);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = lane + 32 * u;
            g[u] = (s < a.n_s && i < n4) ? __ldcs(g4 + i) : make_uint4(0u, 0u, 0u, 0u);
        }
    }
    for (int64_t s = (int64_t)blockIdx.x * nw + wid; s < a.n_s; s += gstride) {
        uint4 gn[U];
        {
            const int64_t sn = s + gstride;
            const uint4* g4n = (const uint4*)(a.G + sn * a.Pst);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = lane + 32 * u;
                gn[u] = (sn < a.n_s && i < n4) ? __ldcs(g4n + i) : make_uint4(0u, 0u, 0u, 0u);
            }
        }
        float t[K], w[K];
#pragma unroll
        for (int kk = 0; kk < K; ++kk) t[kk] = w[kk] = 0.f;
        // correlator lookups issued now, added after the row is consumed
        float cv[kCorrPerLane][K];
        corr_lookups<K>(pb, coff, a.s_cidx + s * a.ncst, a.V, a.invC, lane, cv);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t e[4] = {g[u].x, g[u].y, g[u].z, g[u].w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float val = __uint_as_float(e[j] << 16);
                const int pq = (int)(e[j] >> 16);
#pragma unroll
                for (int kk = 0; kk < K; ++kk) {
                    if (j & 1) w[kk] += val * vpf[pq * K + kk];
                    else t[kk] += val * vpf[pq * K + kk];
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kCorrPerLane; ++j)
#pragma unroll
            for (int kk = 0; kk < K; ++kk) t[kk] += cv[j][kk];
#pragma unroll
        for (int kk = 0; kk < K; ++kk) t[kk] = warp_sum(t[kk] + w[kk]);
        if (lane == 0) {
#pragma unroll
            for (int kk = 0; kk < K; ++kk) a.Tv[s * K + kk] = t[kk] - obv[kk];
            const double c = (double)(t[0] - obv[0]);
            tt += c * c;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) g[u] = gn[u];
    }
    if (K == 1 && a.tt_part) {   // p . S p of a centered product, for CG
        __shared__ double red[32];
        if (lane == 0) red[wid] = tt;
        __syncthreads();
        if (wid == 0) {
            double v = lane < nw ? red[lane] : 0.0;
            v = warp_sum(v);
            if (lane == 0) a.tt_part[blockIdx.x] = v;
        }
    }
}

// one T entry of a parameter's run: acc += W * t_s
template <int K>
__device__ __forceinline__ void scatter_entry(const float* __restrict__ Tv, int64_t s0, uint32_t v, float (&acc)[K]) {
    const float wv = __uint_as_float(v << 16);
    const int64_t t0 = (s0 + (v >> 16)) * K;
#pragma unroll
    for (int kk = 0; kk < K; ++kk) acc[kk] += wv * __ldg(Tv + t0 + kk);
}

// scatter: raw[pq][kk] = sum over samples containing pq of W t_s for the warp's
// pq.  A run is a whole number of kTRun-entry blocks starting on a 512-byte
// boundary (padding entries weigh zero); lane L's 16-byte word of a block
// holds entries L, L + 32, L + 64, L + 96, so each t_s lookup instruction
// covers 32 consecutive entries.  Two blocks (256 entries) per warp in flight.
template <int K>
__device__ __forceinline__ void scatter_T_param(const SortedArgs& a, int pq) {
    const int lane = threadIdx.x & 31;
    float acc[K], acc2[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) acc[kk] = acc2[kk] = 0.f;
    const uint4* T4 = (const uint4*)a.T;
    for (int c = 0; c < a.nchunk; ++c) {
        const uint32_t* base = a.base + (size_t)c * (a.pb.npf + 1);
        const uint32_t q0 = base[pq] >> 2, q1 = base[pq + 1] >> 2;
        const int64_t s0 = (int64_t)c * 65536;
        uint32_t q = q0 + lane;
        for (; q + 32 < q1; q += 64) {
            const uint4 u0 = __ldcs(T4 + q), u1 = __ldcs(T4 + q + 32);
            scatter_entry<K>(a.Tv, s0, u0.x, acc);
            scatter_entry<K>(a.Tv, s0, u0.y, acc2);
            scatter_entry<K>(a.Tv, s0, u0.z, acc);
            scatter_entry<K>(a.Tv, s0, u0.w, acc2);
            scatter_entry<K>(a.Tv, s0, u1.x, acc);
            scatter_entry<K>(a.Tv, s0, u1.y, acc2);
            scatter_entry<K>(a.Tv, s0, u1.z, acc);
            scatter_entry<K>(a.Tv, s0, u1.w, acc2);
        }
        if (q < q1) {
            const uint4 u0 = __ldcs(T4 + q);
            scatter_entry<K>(a.Tv, s0, u0.x, acc);
            scatter_entry<K>(a.Tv, s0, u0.y, acc2);
            scatter_entry<K>(a.Tv, s0, u0.z, acc);
            scatter_entry<K>(a.Tv, s0, u0.w, acc2);
        }
    }
#pragma unroll
    for (int kk = 0; kk < K; ++kk) {
        const float v = warp_sum(acc[kk] + acc2[kk]);
        if (lane == 0) a.raw[(size_t)pq * K + kk] = v;
    }
}

// Both halves of the scatter in one launch: the correlator CTAs first
// (histograms of [0, nhist), or correlator work items of [0, ncb), 8 per CTA,
// a warp per item), then one pairing amplitude per warp.  The short
// correlator CTAs go first so that they do not form a tail behind the long
// pairing runs.
template <int K>
__global__ void __launch_bounds__(256) k_scatter_T(SortedArgs a) {
    if (a.stop && *a.stop) return;
    extern __shared__ __align__(16) unsigned char hist_smem[];
    __shared__ float slots[8][32 * K];
    int b = (int)blockIdx.x;
    if (b < a.nhist) {
        corr_hist_cta<K>(a, b / a.hist_slices, b % a.hist_slices, a.hist_slices, (float*)hist_smem);
        return;
    }
    b -= a.nhist;
    if (b < a.ncb) {
        const int64_t i = (int64_t)b * 8 + (threadIdx.x >> 5);
        if (i < (int64_t)*a.n_items) scatter_C_item<K>(a, a.items[i], slots[threadIdx.x >> 5]);
        return;
    }
    const int pq = (b - a.ncb) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (pq < a.pb.npf) scatter_T_param<K>(a, pq);
}

template __global__ void k_gather_G<1, 1>(SortedArgs);
template __global__ void k_gather_G<1, 2>(SortedArgs);
template __global__ void k_gather_G<1, 3>(SortedArgs);
template __global__ void k_gather_G<1, 4>(SortedArgs);
template __global__ void k_gather_G<1, 5>(SortedArgs);
template __global__ void k_gather_G<1, 6>(SortedArgs);
template __global__ void k_gather_G<1, 7>(SortedArgs);
template __global__ void k_gather_G<1, 8>(SortedArgs);
template __global__ void k_gather_G<1, 9>(SortedArgs);
template __global__ void k_gather_G<1, 10>(SortedArgs);
template __global__ void k_gather_G<1, 11>(SortedArgs);
template __global__ void k_gather_G<1, 12>(SortedArgs);
template __global__ void k_gather_G<1, 13>(SortedArgs);
template __global__ void k_gather_G<1, 14>(SortedArgs);
template __global__ void k_gather_G<1, 15>(SortedArgs);
template __global__ void k_gather_G<1, 16>(SortedArgs);
template __global__ void k_gather_G<2, 4>(SortedArgs);
template __global__ void k_gather_G<2, 8>(SortedArgs);
template __global__ void k_gather_G<2, 16>(SortedArgs);
template __global__ void k_gather_G<4, 4>(SortedArgs);
template __global__ void k_gather_G<4, 8>(SortedArgs);
template __global__ void k_gather_G<4, 16>(SortedArgs);
template __global__ void k_scatter_T<1>(SortedArgs);
template __global__ void k_scatter_T<2>(SortedArgs);
template __global__ void k_scatter_T<4>(SortedArgs);

}  // namespace vmc
