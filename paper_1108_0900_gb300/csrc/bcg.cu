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

// part[blk][4 a + c] = partial sums of U[a] . V[c] over block blk's slice
__global__ void __launch_bounds__(256) k_bcg_gram(const float* U, const float* V, int64_t n, double* part) {
    __shared__ double red[8][16];
    double acc[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) acc[t] = 0.0;
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
            for (int c = 0; c < 4; ++c) acc[4 * a + c] += (double)u[a] * (double)v[c];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        const double s = warp_sum(acc[t]);
        if (lane == 0) red[w][t] = s;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][threadIdx.x];
        part[(int64_t)blockIdx.x * 16 + threadIdx.x] = s;
    }
}

// X += P alpha, R -= Q alpha (alpha 4 x 4 row-major, FP64)
__global__ void __launch_bounds__(256) k_bcg_step(float* X, float* R, const float* P, const float* Q,
                                                  const double* alpha, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float p[4], q[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            p[j] = P[(int64_t)j * n + i];
            q[j] = Q[(int64_t)j * n + i];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double dx = 0.0, dr = 0.0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                dx += (double)p[a] * alpha[4 * a + c];
                dr += (double)q[a] * alpha[4 * a + c];
            }
            X[(int64_t)c * n + i] += (float)dx;
            R[(int64_t)c * n + i] -= (float)dr;
        }
    }
}

// P = R + P beta (beta 4 x 4 row-major, FP64)
__global__ void __launch_bounds__(256) k_bcg_dir(float* P, const float* R, const double* beta, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float p[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) p[j] = P[(int64_t)j * n + i];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double v = (double)R[(int64_t)c * n + i];
#pragma unroll
            for (int a = 0; a < 4; ++a) v += (double)p[a] * beta[4 * a + c];
            P[(int64_t)c * n + i] = (float)v;
        }
    }
}

}  // namespace vmc
