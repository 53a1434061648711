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
//      kTChunk samples (a counting sort of G by pq), each run padded to whole
//      128-entry blocks and interleaved inside a block: the scatter
//      out[pq] = sum_s t_s W_s[pq] sums contiguous runs against the chunk's
//      t_s staged in shared memory, with no atomics and no per-CTA partial
//      images.
//
// The build (count, scan, fill) streams G three times once per SR step.
#include <type_traits>
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
                                                 int wq, int64_t Gst, uint32_t* G, uint16_t* G16, int64_t Gst16) {
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
    if (G16) {   // the compact copy: values only, in the row-major pair order
        uint16_t* d16 = G16 + s * Gst16;
        for (int r = lane; r < Gst16; r += 32) d16[r] = r < P ? src[fulltab[r] & 0xFFFFu] : (uint16_t)0;
    }
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
// length padded to a whole number of kTRun-entry blocks.  Sixteen blocks'
// counts are loaded before they are summed, so a thread waits on one round
// trip per sixteen blocks instead of one per block.
__global__ void k_scan_blocks(uint32_t* counts, int nblk, int npf, uint32_t* total) {
    const int pq = blockIdx.x * blockDim.x + threadIdx.x;
    if (pq >= npf) return;
    constexpr int kAhead = 16;
    uint32_t run = 0u;
    int b = 0;
    for (; b + kAhead <= nblk; b += kAhead) {
        uint32_t c[kAhead];
#pragma unroll
        for (int u = 0; u < kAhead; ++u) c[u] = counts[(size_t)(b + u) * npf + pq];
#pragma unroll
        for (int u = 0; u < kAhead; ++u) {
            counts[(size_t)(b + u) * npf + pq] = run;
            run += c[u];
        }
    }
    for (; b < nblk; ++b) {
        const uint32_t c = counts[(size_t)b * npf + pq];
        counts[(size_t)b * npf + pq] = run;
        run += c;
    }
    total[pq] = (run + kTRun - 1) / kTRun * kTRun;
}

// Position inside a run of logical entry r.  Within each kTRun = 128 entry
// block, entry 32 j + L sits at 4 L + j, so lane L's 16-byte word holds
// entries L, L + 32, L + 64, L + 96 and the j-th lookup instruction of the
// scatter covers 32 consecutive entries (k_rank_T then reorders each block by
// shared-memory bank).
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

// Bank order inside T's blocks, once per set of samples after the fill.
// The scatter's j-th lookup instruction over a block reads t_s for the
// entries at positions 4 L + j (lane L); with the samples in fill order
// their shared-memory banks (s mod 32) collide about 3.5 times per
// instruction.  One warp per 128-entry block sorts the block's entries by
// bank (stable): each bank's entries then sit at consecutive positions and
// go round-robin to the four instructions, about 2.2 wavefronts each.
// Entries of weight zero (the run padding) take the last positions,
// re-pointed at sample (position / 4) mod 32 of the chunk (a staged t_s).
// Only the order inside each block changes: a block holds one parameter's
// entries before and after.
__global__ void __launch_bounds__(256) k_rank_T(uint32_t* T, int64_t t_chunk, int nchunk, const uint32_t* base,
                                                int npf, int64_t n_s) {
    __shared__ uint32_t cnt[8][32];
    __shared__ __align__(16) uint32_t buf[8][kTRun];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t nblk = t_chunk / kTRun, gstep = (int64_t)gridDim.x * 8;
    // block gw of the warp's sequence, or -1 past the chunk's runs; the next
    // block's word is loaded before the current one is sorted
    auto block_start = [&](int64_t gw) -> int64_t {
        if (gw >= nchunk * nblk) return -1;
        const int c = (int)(gw / nblk);
        const int64_t e0 = (int64_t)c * t_chunk + (gw - (int64_t)c * nblk) * kTRun;
        return e0 < (int64_t)__ldg(base + (size_t)c * (npf + 1) + npf) ? e0 : -1;
    };
    int64_t gw = (int64_t)blockIdx.x * 8 + wid;
    int64_t e_next = block_start(gw);
    uint4 w_next = e_next >= 0 ? reinterpret_cast<const uint4*>(T + e_next)[lane] : make_uint4(0u, 0u, 0u, 0u);
    for (; gw < nchunk * nblk; gw += gstep) {
        const int64_t e0 = e_next;
        const uint4 w = w_next;
        e_next = block_start(gw + gstep);
        if (e_next >= 0) w_next = reinterpret_cast<const uint4*>(T + e_next)[lane];
        if (e0 < 0) continue;   // past the chunk's runs
        const int c = (int)(gw / nblk);
        const int ns = (int)min((int64_t)kTChunk, n_s - (int64_t)c * kTChunk);
        uint4* w4 = reinterpret_cast<uint4*>(T + e0);
        const uint32_t e[4] = {w.x, w.y, w.z, w.w};
        cnt[wid][lane] = 0u;
        __syncwarp();
        uint32_t rk[4];
        bool real[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {   // rank of each entry within its bank (block order)
            real[j] = (e[j] & 0xFFFFu) != 0u;
            const uint32_t b = (e[j] >> 16) & 31u;
            const uint32_t peers = __match_any_sync(0xffffffffu, real[j] ? b : 32u + (uint32_t)lane);
            const uint32_t pre = real[j] ? cnt[wid][b] : 0u;
            rk[j] = pre + __popc(peers & lt);
            __syncwarp();
            if (real[j] && (peers & lt) == 0u) cnt[wid][b] = pre + __popc(peers);
            __syncwarp();
        }
        // first position of each bank: exclusive scan of the counts (lane = bank)
        const uint32_t cl = cnt[wid][lane];
        uint32_t incl = cl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        uint32_t free_pos = __shfl_sync(0xffffffffu, incl, 31);   // the real entries
        __syncwarp();
        cnt[wid][lane] = incl - cl;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t fb = __ballot_sync(0xffffffffu, !real[j]);
            uint32_t pos, v = e[j];
            if (real[j]) {
                pos = cnt[wid][(e[j] >> 16) & 31u] + rk[j];
            } else {
                pos = free_pos + __popc(fb & lt);
                const uint32_t sf = (pos >> 2) & 31u;
                v = ((int)sf < ns ? sf : 0u) << 16;
            }
            free_pos += __popc(fb);
            buf[wid][pos] = v;
        }
        __syncwarp();
        w4[lane] = reinterpret_cast<const uint4*>(buf[wid])[lane];
        __syncwarp();
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

// acc += W x[j] for one (j << 16 | bf16 W) entry, x a shared-memory table of K
// floats per index (one 4-, 8- or 16-byte load): the gather's v table
// (j = pq) and the scatter's per-chunk t_s table (j = sample in the chunk)
template <int K>
__device__ __forceinline__ void scatter_entry(const float* tv, uint32_t v, float (&acc)[K]) {
    const float wv = __uint_as_float(v << 16);
    const uint32_t j = v >> 16;
    if constexpr (K == 4) {
        const float4 t = reinterpret_cast<const float4*>(tv)[j];
        acc[0] += wv * t.x; acc[1] += wv * t.y; acc[2] += wv * t.z; acc[3] += wv * t.w;
    } else if constexpr (K == 2) {
        const float2 t = reinterpret_cast<const float2*>(tv)[j];
        acc[0] += wv * t.x; acc[1] += wv * t.y;
    } else {
        acc[0] += wv * tv[j];
    }
}

// gather: t_s = sum_c V[k_c]/C[k_c] + sum_e W_e v[pq(e)] - Obar . V, warp per
// sample.  Centering t_s makes the scatter produce the covariance
// (1/n) sum_s (t_s - Obar . V) O_s = S V directly, with no cancellation
// between <O (O . V)> and Obar (Obar . V).  U = ceil(Pst / 128): every lane
// holds its U 16-byte words of a row, and the warp loads its next row while
// it works on the current one, so a whole row (6 KB at 56 electrons) is
// always in flight per warp.
// rows per warp ahead of the current one whose bulk L2 prefetch the gather
// issues (0: none).  One row ahead, the same row as the register loads that
// follow: one bulk request per row reaches DRAM ahead of the 13 loads per lane
// (measured: 1,380 against 1,354 GB/s per product; two rows ahead 1,341,
// four 1,316)
constexpr int kGatherAhead = 1;

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
        // a bulk L2 request for row s + kGatherAhead gstride (no registers
        // held) ahead of the per-lane loads of the next row below
        if (kGatherAhead > 0 && lane == 0 && s + kGatherAhead * gstride < a.n_s)
            prefetch_l2(a.G + (s + kGatherAhead * gstride) * a.Pst, (uint32_t)(a.Pst * 4));
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
                if (j & 1) scatter_entry<K>(vpf, e[j], w);   // w += W_e v[pq(e)] (K values: one load)
                else scatter_entry<K>(vpf, e[j], t);
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

// Pairing half of the scatter for one chunk c of kTChunk samples and one
// group of pq_per_cta consecutive parameters: raw[pq][kk] (or the chunk's
// partial) = sum over the chunk's samples containing pq of W t_s.
//
// The chunk's t_s (K floats per sample, at most 128 KB) are staged in shared
// memory once per CTA, so every entry's lookup is a shared-memory load
// instead of an L1/L2 round trip.  The group's runs are consecutive in T, and
// each warp takes a consecutive share of the group's parameters, so its
// words form one contiguous stream: the warp keeps NWF blocks of 32 words
// (128 entries, one word per lane) in flight and loads the next NWF blocks
// before it works on the current ones, across run boundaries; the lookups of
// all NWF blocks are issued before their sums.  Every block belongs to one
// parameter (runs are whole blocks, padding entries weigh zero); when a block
// starts past the current run, the warp sums its lanes and writes the
// finished parameter.  Lane L's word of a block holds the block's entries
// 4 L .. 4 L + 3; k_rank_T sorts each block by the bank of its sample, so
// the j-th lookup instruction (entries 4 L + j) meets each bank about twice.
constexpr uint32_t kScatterAhead = 4;   // iterations of the scatter's T stream prefetched into L2

// Correlator half of the scatter for chunk c inside pairing CTA (c, g): for
// every correlator j = g, g + ngrp, ... a shared-memory histogram over j's
// 4^m states of the chunk's staged t_s (states read correlator-major,
// coalesced; t_s in sample order, conflict-free), then each nonzero bin is
// added to craw[corr_off_j + state] (zeroed by the caller) with one vector
// reduction.  Blocks of few states get one copy of the histogram per warp, so
// that fewer lanes add to one address.
template <int K>
__device__ __forceinline__ void chunk_corr_hist(const SortedArgs& a, int c, int g, int ngrp, const float* tv,
                                                float* hist) {
    using TK = typename std::conditional<K == 4, float4, typename std::conditional<K == 2, float2, float>::type>::type;
    const DevProblem& pb = a.pb;
    const int64_t s0 = (int64_t)c * kTChunk;
    const int ns = (int)min((int64_t)kTChunk, a.n_s - s0);
    const int nw = blockDim.x >> 5, wid = threadIdx.x >> 5, bd = blockDim.x;
    const TK* tvk = reinterpret_cast<const TK*>(tv);
    for (int j = g; j < pb.ncorr; j += ngrp) {
        const int d = 1 << (2 * (pb.corr_ptr[j + 1] - pb.corr_ptr[j]));
        const int copies = max(1, min(nw, a.hist_cap / (d * K)));
        float* hw = hist + (size_t)(wid % copies) * d * K;   // [K][d]: one component's bins over all banks
        __syncthreads();   // the previous correlator's bins are read
        for (int i = threadIdx.x; i < copies * d * K; i += bd) hist[i] = 0.f;
        __syncthreads();
        const cstate_t* st = a.cidxT + (int64_t)j * a.n_s + s0;
        int s = threadIdx.x;
        for (; s + 3 * bd < ns; s += 4 * bd) {
            int k[4];
            TK t[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                k[u] = (int)__ldcs(st + s + u * bd);
                t[u] = tvk[s + u * bd];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float* tf = reinterpret_cast<const float*>(&t[u]);
#pragma unroll
                for (int kk = 0; kk < K; ++kk) atomicAdd(&hw[kk * d + k[u]], tf[kk]);
            }
        }
        for (; s < ns; s += bd) {
            const int k = (int)__ldcs(st + s);
            const TK t = tvk[s];
            const float* tf = reinterpret_cast<const float*>(&t);
#pragma unroll
            for (int kk = 0; kk < K; ++kk) atomicAdd(&hw[kk * d + k], tf[kk]);
        }
        __syncthreads();
        float* dst = a.craw + (size_t)pb.corr_off[j] * K;
        for (int i = threadIdx.x; i < d; i += bd) {
            float x[K];
            bool nz = false;
#pragma unroll
            for (int kk = 0; kk < K; ++kk) {
                float v = 0.f;
                for (int cp = 0; cp < copies; ++cp) v += hist[((size_t)cp * K + kk) * d + i];
                x[kk] = v;
                nz |= v != 0.f;
            }
            if (nz) red_add<K>(dst + (size_t)i * K, x);
        }
    }
}

template <int K>
__device__ __forceinline__ void scatter_T_chunk(const SortedArgs& a, int c, int grp, int ngrp, float* tv,
                                                uint32_t* sb, float* hist) {
    constexpr int NWF = 2;
    using TK = typename std::conditional<K == 4, float4, typename std::conditional<K == 2, float2, float>::type>::type;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int npf = a.pb.npf;
    const int p0 = grp * a.pq_per_cta, p1 = min(npf, p0 + a.pq_per_cta);
    const uint32_t* base = a.base + (size_t)c * (npf + 1);
    const int per = (p1 - p0 + nw - 1) / nw;
    const int pa = min(p1, p0 + wid * per), pb = min(p1, pa + per);
    const uint32_t W0 = __ldg(base + pa) >> 2, W1 = __ldg(base + pb) >> 2;   // the warp's words
    const uint4* T4 = (const uint4*)a.T;
    // the stream runs kScatterAhead iterations ahead of the loads as L2
    // prefetches (bytes in flight without registers)
    constexpr uint32_t kStep = 32u * NWF, kAhead = kStep * kScatterAhead;
    if (lane == 0 && W0 < W1) prefetch_l2(T4 + W0, 16u * min(W1 - W0, kAhead + kStep));
    uint4 u[NWF];
#pragma unroll
    for (int i = 0; i < NWF; ++i)
        u[i] = W0 + 32u * i < W1 ? __ldcs(T4 + W0 + 32u * i + lane) : make_uint4(0u, 0u, 0u, 0u);
    // stage the chunk's t_s and the group's run ends (in words) while the
    // first blocks are in flight
    {
        const int64_t s0 = (int64_t)c * kTChunk;
        const int nf = (int)(min((int64_t)kTChunk, a.n_s - s0) * K);
        const float* src = a.Tv + s0 * K;
        for (int i = threadIdx.x; i < nf / 4; i += blockDim.x)
            reinterpret_cast<float4*>(tv)[i] = __ldcg(reinterpret_cast<const float4*>(src) + i);
        for (int i = (nf / 4) * 4 + threadIdx.x; i < nf; i += blockDim.x) tv[i] = __ldcg(src + i);
        for (int i = threadIdx.x; i < p1 - p0; i += blockDim.x) sb[i] = __ldg(base + p0 + i + 1) >> 2;
    }
    __syncthreads();
    const TK* tvk = reinterpret_cast<const TK*>(tv);
    float* out = a.nchunk == 1 ? a.raw : a.part + (size_t)c * npf * K;
    float acc[K], acc2[K];
#pragma unroll
    for (int kk = 0; kk < K; ++kk) acc[kk] = acc2[kk] = 0.f;
    int pq = pa;
    uint32_t pend = pa < pb ? sb[pa - p0] : 0u;   // end of pq's run
    for (uint32_t w = W0; w < W1; w += kStep) {
        const uint32_t wn = w + kStep;
        if (lane == 0 && wn + kAhead < W1) prefetch_l2(T4 + wn + kAhead, 16u * min(W1 - (wn + kAhead), kStep));
        uint4 un[NWF];
#pragma unroll
        for (int i = 0; i < NWF; ++i)
            un[i] = wn + 32u * i < W1 ? __ldcs(T4 + wn + 32u * i + lane) : make_uint4(0u, 0u, 0u, 0u);
        TK x[NWF][4];
#pragma unroll
        for (int i = 0; i < NWF; ++i) {
            x[i][0] = tvk[u[i].x >> 16];
            x[i][1] = tvk[u[i].y >> 16];
            x[i][2] = tvk[u[i].z >> 16];
            x[i][3] = tvk[u[i].w >> 16];
        }
#pragma unroll
        for (int i = 0; i < NWF; ++i) {
            const uint32_t blk = w + 32u * i;
            if (blk < W1) {
                while (blk >= pend) {   // the runs before this block are complete
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        const float v = warp_sum(acc[kk] + acc2[kk]);
                        if (lane == 0) out[(size_t)pq * K + kk] = v;
                        acc[kk] = acc2[kk] = 0.f;
                    }
                    ++pq;
                    pend = sb[pq - p0];
                }
                const uint32_t e[4] = {u[i].x, u[i].y, u[i].z, u[i].w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float wv = __uint_as_float(e[j] << 16);
                    const float* xv = reinterpret_cast<const float*>(&x[i][j]);
#pragma unroll
                    for (int kk = 0; kk < K; ++kk) {
                        if (j & 1) acc2[kk] = fmaf(wv, xv[kk], acc2[kk]);
                        else acc[kk] = fmaf(wv, xv[kk], acc[kk]);
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < NWF; ++i) u[i] = un[i];
    }
    for (; pq < pb; ++pq) {   // the last run, and empty runs after it
#pragma unroll
        for (int kk = 0; kk < K; ++kk) {
            const float v = warp_sum(acc[kk] + acc2[kk]);
            if (lane == 0) out[(size_t)pq * K + kk] = v;
            acc[kk] = acc2[kk] = 0.f;
        }
    }
    if (a.corr_in_cta) chunk_corr_hist<K>(a, c, grp, ngrp, tv, hist);
    if (a.nchunk == 1) return;
    // the last of the group's nchunk CTAs to finish sums the chunks' partials
    // in chunk order (deterministic) and re-arms the group's counter
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(a.done + grp, 1u) == (unsigned)(a.nchunk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int n = (p1 - p0) * K;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float x = 0.f;
        for (int cc = 0; cc < a.nchunk; ++cc) x += __ldcg(a.part + ((size_t)cc * npf + p0) * K + i);
        a.raw[(size_t)p0 * K + i] = x;
    }
    if (threadIdx.x == 0) a.done[grp] = 0u;
}

// The scatter.  Pairing CTA b is chunk b / ngrp and parameter group b % ngrp
// (CTAs of one chunk run together and read its t_s from L2).  The correlator
// half: with a.corr_in_cta, histograms of the chunk's staged t_s built by
// the pairing CTAs after their runs; else shared-memory histograms in CTAs
// [0, nhist) ahead of the pairing CTAs, taking (class, sample slice) =
// (b / hist_slices, b % hist_slices); else correlator work items, as CTAs of
// their own ahead (a.ncb > 0: one item per warp) or after each pairing CTA's
// runs, strided over all warps of the grid.  Dynamic shared memory: the
// chunk's t_s (kTChunk K floats), the group's run ends and the in-CTA
// histograms (from byte hist_off), or a class histogram.
template <int K>
__global__ void __launch_bounds__(scatter_threads(K), scatter_min_ctas(K)) k_scatter_T(SortedArgs a) {
    if (a.stop && *a.stop) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float slots[scatter_threads(K) / 32][32 * K];
    const int nw = blockDim.x >> 5, wid = threadIdx.x >> 5;
    int b = (int)blockIdx.x;
    if (b < a.nhist) {
        corr_hist_cta<K>(a, b / a.hist_slices, b % a.hist_slices, a.hist_slices, (float*)smem);
        return;
    }
    b -= a.nhist;
    if (b < a.ncb) {
        const int64_t i = (int64_t)b * nw + wid;
        if (i < (int64_t)*a.n_items) scatter_C_item<K>(a, a.items[i], slots[wid]);
        return;
    }
    b -= a.ncb;
    const int ngrp = (a.pb.npf + a.pq_per_cta - 1) / a.pq_per_cta;
    float* tv = (float*)smem;
    scatter_T_chunk<K>(a, b / ngrp, b % ngrp, ngrp, tv, (uint32_t*)(tv + (size_t)kTChunk * K),
                       (float*)(smem + a.hist_off));
    if (a.pb.ncorr == 0 || a.ncb > 0 || a.nhist > 0 || a.corr_in_cta) return;
    const int64_t n_items = (int64_t)*a.n_items;
    const int64_t stride = (int64_t)(gridDim.x - a.ncb - a.nhist) * nw;
    for (int64_t i = (int64_t)b * nw + wid; i < n_items; i += stride) scatter_C_item<K>(a, a.items[i], slots[wid]);
}

// Compact gather (one vector): t_s = sum_c V[k_c]/C[k_c] + sum_e W_e v[pq(e)]
// - Obar . V from G16, the sample's 2-byte values in the row-major order of
// electron pairs (a < b), so no index is stored: pq(e) = rowbase(occ[a]) +
// occ[b] comes from the sample's occupation row, which the warp keeps in
// shared memory.  Half the bytes of G per product (3,088 of 6,208 B per
// sample at 56 electrons) for one conflict-free byte lookup per element;
// the v lookups follow the pair order (no bank ranking).  Lane L holds words
// L + 32 u of the row (8 values each) and loads the next sample's words
// before it works on the current ones.  wtab[w] = a | b << 8 is the pair of
// word w's first value; the pair advances along the row (b + 1, or the next
// row a + 1, b = a + 2).  Zero values (the row padding) are skipped.
template <int U>
__global__ void __launch_bounds__(512) k_gather_C(SortedArgs a, const uint16_t* G16, int64_t Gst16,
                                                 const uint16_t* wtab_g, const uint8_t* s_occ, int Nst) {
    if (a.stop && *a.stop) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const DevProblem& pb = a.pb;
    const int nw16 = (int)(Gst16 >> 3);
    const int occ_row = Nst + 16;   // bytes per warp: the row and a zero tail read past its end
    float* vpf = (float*)smem;
    int* coff = (int*)(vpf + pb.npf);
    uint16_t* wtab = (uint16_t*)(coff + pb.ncorr + 1);
    uint8_t* occs = (uint8_t*)(wtab + ((nw16 + 7) & ~7));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < pb.npf; i += blockDim.x) vpf[i] = a.V[pb.ncp + i];
    for (int i = threadIdx.x; i <= pb.ncorr; i += blockDim.x) coff[i] = (int)pb.corr_off[i];
    for (int i = threadIdx.x; i < nw16; i += blockDim.x) wtab[i] = wtab_g[i];
    for (int i = threadIdx.x; i < nw * occ_row; i += blockDim.x) occs[i] = 0;
    __shared__ float obv;
    if (threadIdx.x < 32) {
        const double c = warp_sum_partials(a.obv_part, a.n_obv_part, 0, 1);
        if (threadIdx.x == 0) obv = (float)c;
    }
    __syncthreads();
    uint8_t* occ = occs + wid * occ_row;
    const int M = pb.M, N = pb.N;
    double tt = 0.0;
    const int64_t gstride = (int64_t)gridDim.x * nw;
    const int nocc4 = Nst >> 2;   // 4-byte words of an occupation row
    uint4 g[U];
    uint32_t ow = 0u;
    {
        const int64_t s = (int64_t)blockIdx.x * nw + wid;
        const uint4* g4 = (const uint4*)(G16 + s * Gst16);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = lane + 32 * u;
            g[u] = (s < a.n_s && i < nw16) ? __ldcs(g4 + i) : make_uint4(0u, 0u, 0u, 0u);
        }
        if (s < a.n_s && lane < nocc4) ow = __ldcs((const uint32_t*)(s_occ + s * Nst) + lane);
    }
    for (int64_t s = (int64_t)blockIdx.x * nw + wid; s < a.n_s; s += gstride) {
        __syncwarp();
        if (lane < nocc4) reinterpret_cast<uint32_t*>(occ)[lane] = ow;
        __syncwarp();
        uint4 gn[U];
        {
            const int64_t sn = s + gstride;
            const uint4* g4n = (const uint4*)(G16 + sn * Gst16);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = lane + 32 * u;
                gn[u] = (sn < a.n_s && i < nw16) ? __ldcs(g4n + i) : make_uint4(0u, 0u, 0u, 0u);
            }
            if (sn < a.n_s && lane < nocc4) ow = __ldcs((const uint32_t*)(s_occ + sn * Nst) + lane);
        }
        float cv[kCorrPerLane][1];
        corr_lookups<1>(pb, coff, a.s_cidx + s * a.ncst, a.V, a.invC, lane, cv);
        float t = 0.f, w = 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int wd = lane + 32 * u;
            if (wd < nw16) {
                const uint32_t ab = wtab[wd];
                int ea = (int)(ab & 255u), eb = (int)(ab >> 8);
                int p = occ[ea];
                int rb = p * M - p * (p + 1) / 2 - p - 1;
                const uint32_t e[4] = {g[u].x, g[u].y, g[u].z, g[u].w};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (j > 0 && ++eb == N) {
                        ++ea;
                        eb = ea + 1;
                        p = occ[ea];
                        rb = p * M - p * (p + 1) / 2 - p - 1;
                    }
                    const uint32_t bits = (j & 1) ? (e[j >> 1] >> 16) : (e[j >> 1] & 0xFFFFu);
                    if (bits) {
                        const float x = __uint_as_float(bits << 16) * vpf[rb + occ[eb]];
                        if (j & 1) w += x;
                        else t += x;
                    }
                }
            }
        }
#pragma unroll
        for (int j = 0; j < kCorrPerLane; ++j) t += cv[j][0];
        t = warp_sum(t + w);
        if (lane == 0) {
            a.Tv[s] = t - obv;
            const double c = (double)(t - obv);
            tt += c * c;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) g[u] = gn[u];
    }
    if (a.tt_part) {
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

template __global__ void k_gather_C<4>(SortedArgs, const uint16_t*, int64_t, const uint16_t*, const uint8_t*, int);
template __global__ void k_gather_C<5>(SortedArgs, const uint16_t*, int64_t, const uint16_t*, const uint8_t*, int);
template __global__ void k_gather_C<6>(SortedArgs, const uint16_t*, int64_t, const uint16_t*, const uint8_t*, int);
template __global__ void k_gather_C<7>(SortedArgs, const uint16_t*, int64_t, const uint16_t*, const uint8_t*, int);
template __global__ void k_gather_C<8>(SortedArgs, const uint16_t*, int64_t, const uint16_t*, const uint8_t*, int);
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
template __global__ void k_gather_G<2, 13>(SortedArgs);
template __global__ void k_gather_G<2, 16>(SortedArgs);
template __global__ void k_gather_G<4, 4>(SortedArgs);
template __global__ void k_gather_G<4, 8>(SortedArgs);
template __global__ void k_gather_G<4, 13>(SortedArgs);
template __global__ void k_gather_G<4, 16>(SortedArgs);
template __global__ void k_scatter_T<1>(SortedArgs);
template __global__ void k_scatter_T<2>(SortedArgs);
template __global__ void k_scatter_T<4>(SortedArgs);

}  // namespace vmc
