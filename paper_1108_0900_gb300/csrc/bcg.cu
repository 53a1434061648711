// Enlarged-Krylov block conjugate gradient on (S + eps I) z = b: the
// right-hand side is split into four columns by parameter group (the first
// and second half of the correlators, the same-spin and the opposite-spin
// pairing amplitudes), the four columns advance together as one block CG
// (O'Leary's block recurrences with 4 x 4 step matrices), and z is the sum
// of the columns.  Every iteration is one four-vector S product, which reads
// the O store once for all four columns.  Block vectors are [4][n] FP32,
// column j at offset j n; the 4 x 4 Gram matrices are summed in FP64.
#include "common.cuh"
#include "kernels.h"

namespace vmc {

// B[j][i] = b[i] if parameter i belongs to group j, else 0
__global__ void __launch_bounds__(256) k_bcg_split(const float* b, float* B, int64_t n, int64_t ncp, int64_t corr_split,
                                                   const uint32_t* pq_of, int ns) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int g;
        if (i < ncp) {
            g = i < corr_split ? 0 : 1;
        } else {
            const uint32_t pq = pq_of[i - ncp];
            const int p = (int)(pq & 0xFFFFu), q = (int)(pq >> 16);
            g = ((p < ns) == (q < ns)) ? 2 : 3;
        }
        const float v = b[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) B[(int64_t)j * n + i] = j == g ? v : 0.f;
    }
}

// The iteration runs on the device: Gram partials (exact FP32 products and
// compensated sums per thread, FP64 across threads), one-CTA reductions that
// also solve the 4 x 4
// step systems, and the block updates; every kernel returns at once when
// the stop flag is set (convergence, breakdown or the iteration limit), so
// the host checks the state only every few iterations.

// hi + lo += u v to about FP64 accuracy in FP32 arithmetic: the product's
// rounding error from an FMA (u v = p + e exactly) and the sum's from
// Knuth's two-sum; the rounded intrinsics keep the compiler from fusing them.
// The step systems detect a breakdown by a pivot below 1e-14 of the Gram
// scale, which needs Gram entries this accurate.
__device__ __forceinline__ void acc_exact(float& hi, float& lo, float u, float v) {
    const float p = __fmul_rn(u, v);
    const float e = fmaf(u, v, -p);
    const float s = __fadd_rn(hi, p);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// 16 per-thread (hi, lo) sums -> part[blockIdx.x][16] in FP64 (fixed order)
__device__ __forceinline__ void gram_block_store(const float (&hi)[16], const float (&lo)[16], double* part) {
    __shared__ double red[16][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const double s = warp_sum((double)hi[t] + (double)lo[t]);
        if (lane == 0) red[t][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[threadIdx.x][k];
        part[(int64_t)blockIdx.x * 16 + threadIdx.x] = s;
    }
}

// part[blk][4 a + c] = partial sums of U[a] . V[c] over block blk's slice
__global__ void __launch_bounds__(256) k_bcg_gram(const float* U, const float* V, int64_t n, double* part,
                                                  const int* stop) {
    if (stop && *stop) return;
    float hi[16], lo[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) hi[t] = lo[t] = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float u[4], v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            u[j] = U[(int64_t)j * n + i];
            v[j] = V[(int64_t)j * n + i];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc_exact(hi[4 * a + c], lo[4 * a + c], u[a], v[c]);
    }
    gram_block_store(hi, lo, part);
}

// 4 x 4 system A X = B (row-major) by Gaussian elimination with partial
// pivoting; false if a pivot vanishes relative to the matrix scale
__device__ bool solve4_dev(const double* A_in, const double* B_in, double* X) {
    double A[16], B[16], scale = 0.0;
    for (int i = 0; i < 16; ++i) {
        A[i] = A_in[i];
        B[i] = B_in[i];
        scale = fmax(scale, fabs(A[i]));
    }
    if (!(scale > 0.0) || !isfinite(scale)) return false;
    for (int k = 0; k < 4; ++k) {
        int piv = k;
        for (int i = k + 1; i < 4; ++i)
            if (fabs(A[4 * i + k]) > fabs(A[4 * piv + k])) piv = i;
        if (!(fabs(A[4 * piv + k]) > 1e-14 * scale)) return false;
        if (piv != k)
            for (int j = 0; j < 4; ++j) {
                double t = A[4 * k + j]; A[4 * k + j] = A[4 * piv + j]; A[4 * piv + j] = t;
                t = B[4 * k + j]; B[4 * k + j] = B[4 * piv + j]; B[4 * piv + j] = t;
            }
        for (int i = k + 1; i < 4; ++i) {
            const double f = A[4 * i + k] / A[4 * k + k];
            for (int j = 0; j < 4; ++j) {
                A[4 * i + j] -= f * A[4 * k + j];
                B[4 * i + j] -= f * B[4 * k + j];
            }
        }
    }
    for (int c = 0; c < 4; ++c)
        for (int i = 3; i >= 0; --i) {
            double v = B[4 * i + c];
            for (int j = i + 1; j < 4; ++j) v -= A[4 * i + j] * X[4 * j + c];
            X[4 * i + c] = v / A[4 * i + i];
        }
    return true;
}

// the same, where a block column is exactly zero (a parameter group with no
// right-hand side, e.g. same-spin pairing with one electron per spin): its
// row and column of A and its row of B vanish, so it gets a unit diagonal
// and a zero row in X.  Any other singular A is a breakdown (false).
__device__ bool solve4_reg_dev(const double* A, const double* B, double* X) {
    if (solve4_dev(A, B, X)) return true;
    double Ar[16];
    for (int i = 0; i < 16; ++i) Ar[i] = A[i];
    bool any = false;
    for (int i = 0; i < 4; ++i) {
        bool zero = true;
        for (int j = 0; j < 4; ++j) zero = zero && A[4 * i + j] == 0.0 && A[4 * j + i] == 0.0 && B[4 * i + j] == 0.0;
        if (zero) { Ar[5 * i] = 1.0; any = true; }
    }
    return any && solve4_dev(Ar, B, X);
}

// the 16 sums of nb Gram partials into out (one CTA of 256 threads: 16
// slices of the partials per entry, then the slices in a fixed order)
__device__ __forceinline__ void gram_reduce(const double* part, int nb, double* out) {
    __shared__ double red[16][17];
    const int t = threadIdx.x & 15, sl = threadIdx.x >> 4;
    double s = 0.0;
    for (int b = sl; b < nb; b += 16) s += part[(int64_t)b * 16 + t];
    red[sl][t] = s;
    __syncthreads();
    if (threadIdx.x < 16) {
        double x = 0.0;
        for (int k = 0; k < 16; ++k) x += red[k][threadIdx.x];
        out[threadIdx.x] = x;
    }
    __syncthreads();
}

// start: RR = R^T R, b2 = sum of its entries, thr = itol^2 b2
__global__ void __launch_bounds__(256) k_bcg_start(const double* part, int nb, BcgState* S, double itol) {
    __shared__ double g[16];
    gram_reduce(part, nb, g);
    if (threadIdx.x == 0) {
        double b2 = 0.0;
        for (int i = 0; i < 16; ++i) {
            S->RR[i] = g[i];
            b2 += g[i];
        }
        S->b2 = b2;
        S->thr = itol * itol * b2;
        S->it = 0;
        S->steps = 0;
        S->breakdown = 0;
    }
}

// after Q = A P: alpha = (P^T Q)^{-1} R^T R; a breakdown stops the solve
// before the step
__global__ void __launch_bounds__(256) k_bcg_alpha(const double* part, int nb, BcgState* S, int* stop) {
    if (*stop) return;
    __shared__ double g[16];
    gram_reduce(part, nb, g);
    if (threadIdx.x == 0) {
        ++S->it;
        if (!solve4_reg_dev(g, S->RR, S->al)) {
            S->breakdown = 1;
            *stop = 1;
        }
    }
}

// after the step: RRn = R^T R; stop when sum(RRn) <= itol^2 b2 or at the
// iteration limit, else beta = RR^{-1} RRn and RR = RRn
__global__ void __launch_bounds__(256) k_bcg_beta(const double* part, int nb, BcgState* S, int* stop, int max_iter) {
    if (*stop) return;
    __shared__ double g[16];
    gram_reduce(part, nb, g);
    if (threadIdx.x == 0) {
        ++S->steps;
        double res2 = 0.0;
        for (int i = 0; i < 16; ++i) res2 += g[i];
        if (!isfinite(res2)) {
            S->breakdown = 1;
            *stop = 1;
            return;
        }
        if (res2 <= S->thr || S->it >= max_iter) {
            *stop = 1;
            return;
        }
        if (!solve4_reg_dev(S->RR, g, S->be)) {
            S->breakdown = 1;
            *stop = 1;
            return;
        }
        for (int i = 0; i < 16; ++i) S->RR[i] = g[i];
    }
}

// X += P alpha, R -= Q alpha (alpha from the state, FP32 element arithmetic),
// and the Gram partials of the new R^T R
__global__ void __launch_bounds__(256) k_bcg_step(float* X, float* R, const float* P, const float* Q,
                                                  const BcgState* S, int64_t n, double* part, const int* stop) {
    if (*stop) return;
    float al[16], hi[16], lo[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        al[t] = (float)S->al[t];
        hi[t] = lo[t] = 0.f;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float p[4], q[4], r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            p[j] = P[(int64_t)j * n + i];
            q[j] = Q[(int64_t)j * n + i];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float dx = 0.f, dr = 0.f;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                dx = fmaf(p[a], al[4 * a + c], dx);
                dr = fmaf(q[a], al[4 * a + c], dr);
            }
            X[(int64_t)c * n + i] += dx;
            r[c] = R[(int64_t)c * n + i] - dr;
            R[(int64_t)c * n + i] = r[c];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc_exact(hi[4 * a + c], lo[4 * a + c], r[a], r[c]);
    }
    gram_block_store(hi, lo, part);
}

// P = R + P beta (beta from the state), and the partial dots Obar . P of the
// new directions (part[blk][4], the centering of the next product; the grid
// is the product's partial count)
__global__ void __launch_bounds__(256) k_bcg_dir(float* P, const float* R, const BcgState* S, const double* Obar,
                                                 int64_t n, double* obv_part, const int* stop) {
    if (*stop) return;
    float be[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) be[t] = (float)S->be[t];
    double ob[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float p[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) p[j] = P[(int64_t)j * n + i];
        const double o = Obar[i];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float v = R[(int64_t)c * n + i];
#pragma unroll
            for (int a = 0; a < 4; ++a) v = fmaf(p[a], be[4 * a + c], v);
            P[(int64_t)c * n + i] = v;
            ob[c] += o * (double)v;
        }
    }
    __shared__ double red[4][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const double s = warp_sum(ob[c]);
        if (lane == 0) red[c][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[threadIdx.x][k];
        obv_part[(int64_t)blockIdx.x * 4 + threadIdx.x] = s;
    }
}

}  // namespace vmc
